// Host side of the fast-GFT plan: validation, the stage-by-stage symmetric
// decomposition (Sec. IV-B, IV-C), output ordering, eigenvector signs, the
// 1/sqrt(2) folding, the full FP64 basis, and the device program upload.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>

#include "gft_internal.h"

namespace gft {

namespace {

constexpr double kSymTol = 1e-12;      // phi-symmetry / Laplacian symmetry, x max(1, max|L|)
constexpr double kZeroTol = 1e-12;     // structural zero for component splitting, same scale
constexpr double kClusterTol = 1e-9;   // eigenvalue clusters, x max(1, max|lambda|)
constexpr double kSignTol = 1e-8;      // sign rule: entries below this fraction of max|u| count as zeros
const double kRsqrt2 = 0.70710678118654752440;

double max_abs(const std::vector<double>& v) {
    double m = 0.0;
    for (double x : v) m = std::max(m, std::fabs(x));
    return m;
}

// Connected components of the graph of nonzero off-diagonal entries of an
// m x m matrix; each component ascending, components by smallest index.
std::vector<std::vector<int>> components(const std::vector<double>& A, int m, double tol) {
    std::vector<int> comp(m, -1);
    std::vector<std::vector<int>> out;
    for (int r = 0; r < m; ++r) {
        if (comp[r] >= 0) continue;
        int id = (int)out.size();
        out.emplace_back();
        std::vector<int> stack{r};
        comp[r] = id;
        while (!stack.empty()) {
            int v = stack.back();
            stack.pop_back();
            out[id].push_back(v);
            for (int u = 0; u < m; ++u)
                if (u != v && comp[u] < 0 && std::fabs(A[(size_t)v * m + u]) > tol) {
                    comp[u] = id;
                    stack.push_back(u);
                }
        }
        std::sort(out[id].begin(), out[id].end());
    }
    return out;
}

}  // namespace

std::vector<int> output_positions(const std::vector<double>& lam, const std::vector<int>& leaf,
                                  const std::vector<int>& local) {
    const int N = (int)lam.size();
    double lmax = 0.0;
    for (double v : lam) lmax = std::max(lmax, std::fabs(v));
    const double tol = kClusterTol * std::max(1.0, lmax);
    std::vector<int> idx(N);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return lam[a] < lam[b]; });
    std::vector<int> order;
    int start = 0;
    for (int j = 1; j <= N; ++j) {
        if (j == N || lam[idx[j]] - lam[idx[j - 1]] > tol) {
            std::vector<int> cl(idx.begin() + start, idx.begin() + j);
            std::sort(cl.begin(), cl.end(), [&](int a, int b) {
                return leaf[a] != leaf[b] ? leaf[a] < leaf[b] : local[a] < local[b];
            });
            order.insert(order.end(), cl.begin(), cl.end());
            start = j;
        }
    }
    std::vector<int> pos(N);
    for (int q = 0; q < N; ++q) pos[order[q]] = q;
    return pos;
}

int leaf_bucket(int m) {
    static const int b[] = {4, 8, 16, 24, 32, 48, 64};
    for (int v : b)
        if (m <= v) return v;
    return 0;
}

void analyze(gft_plan_s& p, const double* Lin, int n_stages, const int32_t* phi) {
    const int n = p.n;
    p.L.assign(Lin, Lin + (size_t)n * n);
    for (double v : p.L)
        if (!std::isfinite(v)) fail(GFT_ERR_NOT_LAPLACIAN, "L has a non-finite entry");
    const double scale = std::max(1.0, max_abs(p.L));
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (std::fabs(p.L[(size_t)i * n + j] - p.L[(size_t)j * n + i]) > kSymTol * scale)
                fail(GFT_ERR_NOT_LAPLACIAN, "L is not symmetric at (" + std::to_string(i) + "," +
                                                std::to_string(j) + ")");
    // Definition 1 for every stage
    for (int s = 0; s < n_stages; ++s) {
        const int32_t* f = phi + (size_t)s * n;
        for (int i = 0; i < n; ++i) {
            if (f[i] < 0 || f[i] >= n || f[(int)f[i]] != i)
                fail(GFT_ERR_NOT_INVOLUTION, "stage " + std::to_string(s) +
                                                 ": phi is not an involution at node " +
                                                 std::to_string(i));
        }
    }
    p.n_stages = n_stages;
    std::vector<Leaf> blocks(1);
    blocks[0].labels.resize(n);
    std::iota(blocks[0].labels.begin(), blocks[0].labels.end(), 0);
    blocks[0].L = p.L;
    blocks[0].exps.assign(n, 0);
    p.stages.assign(n_stages, {});

    std::vector<int> pos(n, -1);
    for (int s = 0; s < n_stages; ++s) {
        const int32_t* f = phi + (size_t)s * n;
        std::vector<Leaf> next;
        for (Leaf& b : blocks) {
            const int m = b.m();
            for (int k = 0; k < m; ++k) pos[b.labels[k]] = k;
            std::vector<int> loc(m);
            bool moves = false;
            for (int k = 0; k < m; ++k) {
                int img = pos[f[b.labels[k]]];
                if (img < 0 || b.labels[img] != f[b.labels[k]])
                    fail(GFT_ERR_BLOCK_LEAK, "stage " + std::to_string(s) + ": phi maps node " +
                                                 std::to_string(b.labels[k]) +
                                                 " out of its block '" + b.tag + "'");
                loc[k] = img;
                moves |= (img != k);
            }
            for (int k = 0; k < m; ++k) pos[b.labels[k]] = -1;
            if (!moves) {
                next.push_back(std::move(b));
                continue;
            }
            // Definition 2 on the block Laplacian: l_kl = l_loc(k) loc(l)
            for (int k = 0; k < m; ++k)
                for (int l = 0; l < m; ++l)
                    if (std::fabs(b.L[(size_t)k * m + l] - b.L[(size_t)loc[k] * m + loc[l]]) >
                        kSymTol * scale)
                        fail(GFT_ERR_NOT_SYMMETRIC, "stage " + std::to_string(s) + ": block '" +
                                                        b.tag + "' is not phi-symmetric");
            std::vector<int> X, Z, Y;
            for (int k = 0; k < m; ++k) {
                if (loc[k] > k) X.push_back(k);
                else if (loc[k] == k) Z.push_back(k);
            }
            for (int x : X) Y.push_back(loc[x]);
            for (size_t a = 0; a < X.size(); ++a)
                if (b.exps[X[a]] != b.exps[Y[a]])
                    fail(GFT_ERR_UNSUPPORTED,
                         "stage " + std::to_string(s) + ": nodes " + std::to_string(b.labels[X[a]]) +
                             " and " + std::to_string(b.labels[Y[a]]) +
                             " took part in different numbers of earlier stages");
            // G+ on X then Z, G- on the partners of X (block form of Eq. 17
            // written for B_phi of Eq. 20)
            Leaf plus, minus;
            std::vector<int> P(X);
            P.insert(P.end(), Z.begin(), Z.end());
            const int mp = (int)P.size(), mm = (int)X.size();
            const double sq2 = std::sqrt(2.0);
            auto Lb = [&](int i, int j) { return b.L[(size_t)i * m + j]; };
            plus.L.assign((size_t)mp * mp, 0.0);
            for (int a = 0; a < mp; ++a) {
                const bool ax = a < mm;
                for (int c = 0; c < mp; ++c) {
                    const bool cx = c < mm;
                    double v;
                    if (ax && cx) v = Lb(P[a], P[c]) + Lb(P[a], loc[P[c]]);
                    else if (!ax && !cx) v = Lb(P[a], P[c]);
                    else v = sq2 * Lb(P[a], P[c]);
                    plus.L[(size_t)a * mp + c] = v;
                }
            }
            minus.L.assign((size_t)mm * mm, 0.0);
            for (int a = 0; a < mm; ++a)
                for (int c = 0; c < mm; ++c)
                    minus.L[(size_t)a * mm + c] = Lb(Y[a], Y[c]) - Lb(Y[a], X[c]);
            for (int k : P) {
                plus.labels.push_back(b.labels[k]);
                plus.exps.push_back(b.exps[k] + (loc[k] != k ? 1 : 0));
            }
            for (int k : Y) {
                minus.labels.push_back(b.labels[k]);
                minus.exps.push_back(b.exps[k] + 1);
            }
            plus.tag = b.tag + "+";
            minus.tag = b.tag + "-";
            for (size_t a = 0; a < X.size(); ++a)
                p.stages[s].push_back({b.labels[X[a]], b.labels[Y[a]]});
            next.push_back(std::move(plus));
            next.push_back(std::move(minus));
        }
        blocks.swap(next);
    }
    if (p.flags & GFT_SPLIT_COMPONENTS) {
        std::vector<Leaf> split;
        for (Leaf& b : blocks) {
            const int m = b.m();
            auto comps = components(b.L, m, kZeroTol * scale);
            if (comps.size() == 1) {
                split.push_back(std::move(b));
                continue;
            }
            for (size_t ci = 0; ci < comps.size(); ++ci) {
                Leaf c;
                const auto& cm = comps[ci];
                const int q = (int)cm.size();
                c.L.resize((size_t)q * q);
                for (int a = 0; a < q; ++a) {
                    c.labels.push_back(b.labels[cm[a]]);
                    c.exps.push_back(b.exps[cm[a]]);
                    for (int d = 0; d < q; ++d) c.L[(size_t)a * q + d] = b.L[(size_t)cm[a] * m + cm[d]];
                }
                c.tag = b.tag + "." + std::to_string(ci);
                split.push_back(std::move(c));
            }
        }
        blocks.swap(split);
    }
    p.leaves = std::move(blocks);
}

// Full-length basis vector of leaf k's eigenvector c: U = B_1 ... B_S e,
// with every B_s applied as Eq. 20 ((a+b)/sqrt2 at X, (a-b)/sqrt2 at Y).
static void full_column(const gft_plan_s& p, int k, int c, std::vector<double>& v) {
    const Leaf& lf = p.leaves[k];
    const int m = lf.m();
    v.assign(p.n, 0.0);
    if (p.right && c < (int)p.rpairs.size()) {
        // right Haar unit c: (e_c; f_c)/sqrt2 in E's slot, (e_c; -f_c)/sqrt2 in F's (Eq. 9)
        const Leaf& E = p.leaves[0];
        const Leaf& F = p.leaves[1];
        const double sf = k == 0 ? kRsqrt2 : -kRsqrt2;
        for (int r = 0; r < E.m(); ++r) v[E.labels[r]] = kRsqrt2 * E.V[(size_t)r * E.m() + c];
        for (int r = 0; r < F.m(); ++r) v[F.labels[r]] = sf * F.V[(size_t)r * F.m() + c];
        return;
    }
    for (int r = 0; r < m; ++r) v[lf.labels[r]] = lf.V[(size_t)r * m + c];
    for (int s = p.n_stages - 1; s >= 0; --s)
        for (auto& pr : p.stages[s]) {
            double a = v[pr.first], b = v[pr.second];
            v[pr.first] = (a + b) * kRsqrt2;
            v[pr.second] = (a - b) * kRsqrt2;
        }
}

void compute_basis(const gft_plan_s& p, double* U) {
    const int n = p.n;
    std::vector<double> v;
    int i = 0;
    for (size_t k = 0; k < p.leaves.size(); ++k)
        for (int c = 0; c < p.leaves[k].m(); ++c, ++i) {
            full_column(p, (int)k, c, v);
            const int col = p.out_pos[i];
            for (int r = 0; r < n; ++r) U[(size_t)r * n + col] = v[r];
        }
}

void free_device(gft_plan_s& p) {
    jit_free(p);
    tc_free(p);
    tcn_free(p);
    wide_free(p);
    if (p.dev.d_ints) cudaFree(p.dev.d_ints);
    if (p.dev.d_mats32) cudaFree(p.dev.d_mats32);
    if (p.dev.d_mats64) cudaFree(p.dev.d_mats64);
    if (p.dev.d_nm) cudaFree(p.dev.d_nm);
    if (p.dev.d_err) cudaFree(p.dev.d_err);
    p.dev = DevProgram{};
    for (int b = 0; b < gft_plan_s::kHostStreams; ++b) {
        if (p.d_stage[b]) cudaFree(p.d_stage[b]);
        if (p.d_stage_out[b]) cudaFree(p.d_stage_out[b]);
        if (p.host_streams[b]) cudaStreamDestroy(p.host_streams[b]);
        for (cudaEvent_t* e : {&p.ev_up[b], &p.ev_k[b], &p.ev_down[b]})
            if (*e) {
                cudaEventDestroy(*e);
                *e = nullptr;
            }
        p.d_stage[b] = p.d_stage_out[b] = nullptr;
        p.host_streams[b] = nullptr;
    }
    p.stage_elems = 0;
}

void finalize_host(gft_plan_s& p) {
    const int n = p.n;
    // ---- output order: ascending eigenvalue, clusters by (leaf, index) ----
    std::vector<double> lam_e;
    std::vector<int> leaf_e, local_e;
    for (size_t k = 0; k < p.leaves.size(); ++k)
        for (int c = 0; c < p.leaves[k].m(); ++c) {
            lam_e.push_back(p.leaves[k].lam[c]);
            leaf_e.push_back((int)k);
            local_e.push_back(c);
        }
    const int N = (int)lam_e.size();
    if (p.flags & GFT_ORDER_BLOCK) {
        p.out_pos.assign(N, 0);
        std::iota(p.out_pos.begin(), p.out_pos.end(), 0);
    } else {
        p.out_pos = output_positions(lam_e, leaf_e, local_e);
    }
    // ---- signs: first significant entry (|u_i| > 1e-8 max|u|) of each full
    // vector positive, the convention of the closed forms the paper quotes
    // (DCT-II, the printed 4-cycle basis of Sec. III) ----
    // (right Haar units: the rule fixes the sum vector, i.e. E's column and
    // F's column together; the difference vector follows)
    std::vector<double> v;
    for (size_t k = 0; k < p.leaves.size(); ++k) {
        Leaf& lf = p.leaves[k];
        const int m = lf.m();
        for (int c = 0; c < m; ++c) {
            if (p.right && k == 1) break;
            full_column(p, (int)k, c, v);
            double mx = 0.0;
            for (double x : v) mx = std::max(mx, std::fabs(x));
            const double thr = kSignTol * mx;
            int first = 0;
            while (first < n && !(std::fabs(v[first]) > thr)) ++first;
            if (first < n && v[first] < 0) {
                for (int r = 0; r < m; ++r) lf.V[(size_t)r * m + c] = -lf.V[(size_t)r * m + c];
                if (p.right && c < (int)p.rpairs.size()) {
                    Leaf& F = p.leaves[1];
                    for (int r = 0; r < F.m(); ++r) F.V[(size_t)r * F.m() + c] = -F.V[(size_t)r * F.m() + c];
                }
            }
        }
    }
    p.lam_out.assign(n, 0.0);
    for (int q = 0; q < N; ++q) p.lam_out[p.out_pos[q]] = lam_e[q];
}

void upload_plan(gft_plan_s& p) {
    const int n = p.n;
    DevProgram& d = p.dev;
    d.n = n;
    d.n_leaves = (int)p.leaves.size();
    d.n_pre_stages = p.n_stages;
    d.n_pre_pairs = 0;
    for (auto& st : p.stages) d.n_pre_pairs += (int)st.size();
    // device stages: the left stages, then (bipartite plans) the right
    // Haar units as one more stage over the leaf output slots
    std::vector<std::vector<std::pair<int, int>>> dst(p.stages);
    if (p.right) dst.push_back(p.rpairs);
    d.n_stages = (int)dst.size();
    d.n_pairs = 0;
    for (auto& st : dst) d.n_pairs += (int)st.size();
    std::vector<int> ints;
    for (auto& st : dst)
        for (auto& pr : st) {
            ints.push_back(pr.first);
            ints.push_back(pr.second);
        }
    int acc = 0;
    ints.push_back(0);
    for (auto& st : dst) {
        acc += (int)st.size();
        ints.push_back(acc);
    }
    for (auto& lf : p.leaves) ints.insert(ints.end(), lf.labels.begin(), lf.labels.end());
    ints.insert(ints.end(), p.out_pos.begin(), p.out_pos.end());
    {
        // src[j]: the tile slot holding coefficient j once every leaf has
        // written its outputs over its own input slots (its node labels)
        std::vector<int> src(n, 0);
        int i = 0;
        for (auto& lf : p.leaves)
            for (int c = 0; c < lf.m(); ++c, ++i) src[p.out_pos[i]] = lf.labels[c];
        ints.insert(ints.end(), src.begin(), src.end());
    }
    std::vector<double> mats;
    int off = 0, off_s = 0;
    d.max_bucket = 0;
    bool core_ok = true;
    for (auto& lf : p.leaves) {
        const int m = lf.m(), bk = leaf_bucket(m);
        ints.push_back(m);
        ints.push_back(bk);
        ints.push_back(off);
        ints.push_back((int)mats.size());
        ints.push_back(off_s);
        off += m;
        off_s += bk * bk;
        if (bk == 0) {
            core_ok = false;
            continue;
        }
        d.max_bucket = std::max(d.max_bucket, bk);
        std::vector<double> Mf((size_t)bk * bk, 0.0), Mi((size_t)bk * bk, 0.0);
        for (int r = 0; r < m; ++r) {
            for (int c = 0; c < m; ++c) {
                const double val = lf.fold(r, c);
                Mf[(size_t)r * bk + c] = val;
                Mi[(size_t)c * bk + r] = val;
            }
        }
        mats.insert(mats.end(), Mf.begin(), Mf.end());
        mats.insert(mats.end(), Mi.begin(), Mi.end());
    }
    if (!core_ok) d.max_bucket = 0;  // CUDA-core kernels cannot run this plan
    d.mats_smem = off_s;
    d.ints_count = (int)ints.size();
    d.mats_count = (int)mats.size();
    std::vector<float> mats32(mats.begin(), mats.end());
    GFT_CUDA(cudaMalloc(&d.d_ints, sizeof(int) * std::max<size_t>(1, ints.size())));
    GFT_CUDA(cudaMemcpy(d.d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice));
    if (!mats.empty()) {
        GFT_CUDA(cudaMalloc(&d.d_mats32, sizeof(float) * mats32.size()));
        GFT_CUDA(cudaMemcpy(d.d_mats32, mats32.data(), sizeof(float) * mats32.size(), cudaMemcpyHostToDevice));
        GFT_CUDA(cudaMalloc(&d.d_mats64, sizeof(double) * mats.size()));
        GFT_CUDA(cudaMemcpy(d.d_mats64, mats.data(), sizeof(double) * mats.size(), cudaMemcpyHostToDevice));
    }
    if (core_ok) {
        // node-major program image: [ints][(leaf, 4-output group) list], each
        // part padded to 4 words, so that one run of 16-byte copies brings it in
        std::vector<int32_t> img(ints.begin(), ints.end());
        img.resize((img.size() + 3) & ~size_t(3), 0);
        d.nm_cg_off = (int)img.size();
        d.nm_n_cg = 0;
        for (size_t k = 0; k < p.leaves.size(); ++k)
            for (int c0 = 0; c0 < p.leaves[k].m(); c0 += 4, ++d.nm_n_cg) img.push_back((int32_t)((k << 16) | c0));
        img.resize((img.size() + 3) & ~size_t(3), 0);
        d.nm_words = (int)img.size();
        GFT_CUDA(cudaMalloc(&d.d_nm, sizeof(int32_t) * img.size()));
        GFT_CUDA(cudaMemcpy(d.d_nm, img.data(), sizeof(int32_t) * img.size(), cudaMemcpyHostToDevice));
    }
    GFT_CUDA(cudaMalloc(&d.d_err, sizeof(int)));
    GFT_CUDA(cudaMemset(d.d_err, 0, sizeof(int)));
    p.has_device = true;
}

ApplyArgs apply_args(const gft_plan_s& p, bool f64) {
    ApplyArgs a;
    a.ints = p.dev.d_ints;
    a.mats = f64 ? (const void*)p.dev.d_mats64 : (const void*)p.dev.d_mats32;
    a.n = p.dev.n;
    a.n_stages = p.dev.n_stages;
    a.n_leaves = p.dev.n_leaves;
    a.n_pairs = p.dev.n_pairs;
    a.n_pre_pairs = p.dev.n_pre_pairs;
    a.max_bucket = p.dev.max_bucket;
    a.ints_count = p.dev.ints_count;
    a.mats_count = p.dev.mats_count;
    a.mats_smem = p.dev.mats_smem;
    a.err = p.dev.d_err;
    return a;
}

}  // namespace gft

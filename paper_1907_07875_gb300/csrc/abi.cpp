// extern "C" entry points for plans (include/gft.h).  Every call validates
// its arguments, converts internal exceptions into gft_status codes, and
// records the message for gft_last_error().
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <atomic>
#include <exception>
#include <string>
#include <thread>
#include <vector>

#include "gft_internal.h"

namespace gft {

namespace {
thread_local std::string g_last_error;
}

void fail(gft_status code, const std::string& msg) { throw GftError{code, msg}; }

void set_last_error(const std::string& msg) { g_last_error = msg; }

void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) fail(GFT_ERR_OOM, std::string(what) + ": out of device memory");
    fail(GFT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class F>
gft_status guard(F&& f) {
    try {
        f();
        return GFT_OK;
    } catch (const GftError& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return GFT_ERR_OOM;
    } catch (...) {
        set_last_error("unexpected internal exception");
        return GFT_ERR_INVALID_ARG;
    }
}

const char* last_error_cstr() { return g_last_error.c_str(); }

void check_plan(const gft_plan_s* p) {
    if (!p) fail(GFT_ERR_INVALID_ARG, "plan is NULL");
}

void check_device_plan(const gft_plan_s* p) {
    check_plan(p);
    if (!p->has_device) fail(GFT_ERR_NO_DEVICE, "plan was created with GFT_ANALYZE_ONLY");
}

void check_symmetric_finite(int n, const double* L) {
    double mx = 0.0;
    for (size_t e = 0; e < (size_t)n * n; ++e) {
        if (!std::isfinite(L[e])) fail(GFT_ERR_NOT_LAPLACIAN, "L has a non-finite entry");
        mx = std::max(mx, std::fabs(L[e]));
    }
    const double tol = 1e-12 * std::max(1.0, mx);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (std::fabs(L[(size_t)i * n + j] - L[(size_t)j * n + i]) > tol)
                fail(GFT_ERR_NOT_LAPLACIAN, "L is not symmetric");
}

void check_io(const void* a, const void* b, int64_t batch) {
    if (batch < 0) fail(GFT_ERR_INVALID_ARG, "batch < 0");
    if (batch == 0) return;
    if (!a || !b) fail(GFT_ERR_INVALID_ARG, "NULL signal pointer");
    if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u)
        fail(GFT_ERR_MISALIGNED, "signal pointers must be 16-byte aligned");
}

}  // namespace gft

gft_plan_s::~gft_plan_s() { gft::free_device(*this); }

using namespace gft;

extern "C" {

const char* gft_status_string(gft_status s) {
    switch (s) {
        case GFT_OK: return "GFT_OK";
        case GFT_ERR_INVALID_ARG: return "GFT_ERR_INVALID_ARG";
        case GFT_ERR_NOT_INVOLUTION: return "GFT_ERR_NOT_INVOLUTION";
        case GFT_ERR_NOT_SYMMETRIC: return "GFT_ERR_NOT_SYMMETRIC";
        case GFT_ERR_NOT_LAPLACIAN: return "GFT_ERR_NOT_LAPLACIAN";
        case GFT_ERR_NO_CONVERGENCE: return "GFT_ERR_NO_CONVERGENCE";
        case GFT_ERR_CUDA: return "GFT_ERR_CUDA";
        case GFT_ERR_OOM: return "GFT_ERR_OOM";
        case GFT_ERR_TIMEOUT: return "GFT_ERR_TIMEOUT";
        case GFT_ERR_UNSUPPORTED: return "GFT_ERR_UNSUPPORTED";
        case GFT_ERR_MISALIGNED: return "GFT_ERR_MISALIGNED";
        case GFT_ERR_BLOCK_LEAK: return "GFT_ERR_BLOCK_LEAK";
        case GFT_ERR_NO_DEVICE: return "GFT_ERR_NO_DEVICE";
        case GFT_ERR_NOT_BIPARTITE: return "GFT_ERR_NOT_BIPARTITE";
    }
    return "GFT_ERR_UNKNOWN";
}

const char* gft_last_error(void) { return last_error_cstr(); }

int32_t gft_version(void) { return 10000; }

gft_status gft_laplacian_from_weights(int32_t n, const double* W, const double* s, double* L) {
    return guard([&] {
        if (n < 1 || !W || !L) fail(GFT_ERR_INVALID_ARG, "n < 1 or NULL W / L");
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double w = W[(size_t)i * n + j];
                if (!std::isfinite(w)) fail(GFT_ERR_NOT_LAPLACIAN, "non-finite weight");
                if (i != j && w != W[(size_t)j * n + i]) fail(GFT_ERR_NOT_LAPLACIAN, "W is not symmetric");
            }
        if (s)
            for (int i = 0; i < n; ++i)
                if (!std::isfinite(s[i])) fail(GFT_ERR_NOT_LAPLACIAN, "non-finite self-loop");
        for (int i = 0; i < n; ++i) {
            double d = s ? s[i] : 0.0;
            for (int j = 0; j < n; ++j)
                if (j != i) {
                    d += W[(size_t)i * n + j];
                    L[(size_t)i * n + j] = -W[(size_t)i * n + j];
                }
            L[(size_t)i * n + i] = d;
        }
    });
}

gft_status gft_normalized_laplacian_from_weights(int32_t n, const double* W, const double* s, double* L) {
    return guard([&] {
        const gft_status st = gft_laplacian_from_weights(n, W, s, L);
        if (st != GFT_OK) fail(st, last_error_cstr());
        // D^-1/2 L D^-1/2 with d_i = l_ii (the degree, self-loop included)
        std::vector<double> r(n);
        for (int i = 0; i < n; ++i) {
            const double d = L[(size_t)i * n + i];
            if (!(d > 0.0)) fail(GFT_ERR_NOT_LAPLACIAN, "node " + std::to_string(i) + " has no positive degree");
            r[i] = 1.0 / std::sqrt(d);
        }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) L[(size_t)i * n + j] = (L[(size_t)i * n + j] * r[i]) * r[j];
    });
}

}  // extern "C"

namespace gft {
namespace {

void check_create_args(int32_t n, const double* L, int32_t n_stages, const int32_t* phi, uint32_t flags) {
    if (n < 1 || n > 4096) fail(GFT_ERR_INVALID_ARG, "n must be in [1, 4096]");
    if (!L) fail(GFT_ERR_INVALID_ARG, "L is NULL");
    if (n_stages < 0 || n_stages > 16) fail(GFT_ERR_INVALID_ARG, "n_stages must be in [0, 16]");
    if (n_stages > 0 && !phi) fail(GFT_ERR_INVALID_ARG, "phi is NULL");
    if (flags & ~(GFT_SPLIT_COMPONENTS | GFT_ORDER_BLOCK | GFT_ANALYZE_ONLY | GFT_NO_JIT | GFT_KERNEL_TABLE |
                  GFT_KERNEL_WIDE | GFT_SEARCH_STAGES | GFT_NORMALIZED))
        fail(GFT_ERR_INVALID_ARG, "unknown flag");
    if ((flags & GFT_KERNEL_TABLE) && (flags & GFT_KERNEL_WIDE))
        fail(GFT_ERR_INVALID_ARG, "GFT_KERNEL_TABLE and GFT_KERNEL_WIDE are exclusive");
    if ((flags & GFT_SEARCH_STAGES) && n_stages != 0)
        fail(GFT_ERR_INVALID_ARG, "GFT_SEARCH_STAGES finds the stages: pass n_stages = 0");
}

// D^-1/2 L D^-1/2 with d_i = l_ii (Sec. II-B), as gft_normalized_laplacian_from_weights
std::vector<double> normalized_copy(int n, const double* L) {
    std::vector<double> N(L, L + (size_t)n * n), r(n);
    for (int i = 0; i < n; ++i) {
        const double d = L[(size_t)i * n + i];
        if (!(d > 0.0) || !std::isfinite(d))
            fail(GFT_ERR_NOT_LAPLACIAN, "node " + std::to_string(i) + " has no positive degree");
        r[i] = 1.0 / std::sqrt(d);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) N[(size_t)i * n + j] = (N[(size_t)i * n + j] * r[i]) * r[j];
    return N;
}

// Decompose every graph on the host, eigendecompose all their leaves in one
// batched Jacobi solve on the device, then finish and upload each plan.
void create_plans(int32_t count, const int32_t* ns, const double* const* Ls, const int32_t* n_stages,
                  const int32_t* const* phis, uint32_t flags, gft_plan_t* out) {
    for (int i = 0; i < count; ++i)
        check_create_args(ns[i], Ls[i], n_stages[i], phis ? phis[i] : nullptr, flags);
    std::vector<std::unique_ptr<gft_plan_s>> made(count);
    for (int i = 0; i < count; ++i) {
        made[i].reset(new gft_plan_s);
        made[i]->n = ns[i];
        made[i]->flags = flags;
    }
    // host decomposition: independent per graph, spread over host threads
    // (largest graphs first); the first failing graph in input order decides
    // the error, as in a sequential run
    {
        std::vector<int> order(count);
        for (int i = 0; i < count; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ns[a] > ns[b]; });
        std::vector<std::exception_ptr> errs(count);
        std::atomic<int> next{0};
        auto work = [&] {
            for (int q = next++; q < count; q = next++) {
                const int i = order[q];
                try {
                    const int n = ns[i];
                    std::vector<double> Ln;
                    const double* L = Ls[i];
                    if (flags & GFT_NORMALIZED) {
                        Ln = normalized_copy(n, L);
                        L = Ln.data();
                    }
                    if (flags & GFT_SEARCH_STAGES) {
                        check_symmetric_finite(n, L);
                        std::vector<int> found;
                        const int s = search_stages(n, L, 16, 1000000, found);
                        analyze(*made[i], L, s, found.data());
                    } else {
                        analyze(*made[i], L, n_stages[i], phis ? phis[i] : nullptr);
                    }
                } catch (...) {
                    errs[i] = std::current_exception();
                }
            }
        };
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        const int nt = std::min({hw, 16, std::max(1, count / 8)});
        std::vector<std::thread> pool;
        for (int t = 1; t < nt; ++t) pool.emplace_back(work);
        work();
        for (auto& th : pool) th.join();
        for (int i = 0; i < count; ++i)
            if (errs[i]) std::rethrow_exception(errs[i]);
    }
    if (!(flags & GFT_ANALYZE_ONLY)) {
        int dev = 0;
        GFT_CUDA(cudaGetDevice(&dev));
        std::vector<Leaf*> all;
        for (auto& p : made) {
            p->device = dev;
            for (auto& lf : p->leaves) all.push_back(&lf);
        }
        cudaStream_t st = nullptr;
        GFT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        try {
            jacobi_leaf_ptrs(all, st);
        } catch (...) {
            cudaStreamDestroy(st);
            throw;
        }
        GFT_CUDA(cudaStreamDestroy(st));
        for (auto& p : made) {
            finalize_host(*p);
            upload_plan(*p);
            jit_build(*p);
            wide_build(*p);
        }
        GFT_CUDA(cudaDeviceSynchronize());
    }
    for (int i = 0; i < count; ++i) out[i] = made[i].release();
}

}  // namespace
}  // namespace gft

extern "C" {

gft_status gft_plan_create(int32_t n, const double* L, int32_t n_stages, const int32_t* phi,
                           uint32_t flags, gft_plan_t* out) {
    return guard([&] {
        if (!out) fail(GFT_ERR_INVALID_ARG, "out is NULL");
        const int32_t* phis[1] = {phi};
        create_plans(1, &n, &L, &n_stages, phis, flags, out);
    });
}

gft_status gft_plan_create_many(int32_t count, const int32_t* n, const double* const* L,
                                const int32_t* n_stages, const int32_t* const* phi, uint32_t flags,
                                gft_plan_t* out) {
    return guard([&] {
        if (!out || !n || !L || !n_stages) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        if (count < 0) fail(GFT_ERR_INVALID_ARG, "count < 0");
        if (count == 0) return;
        bool any_stage = false;
        for (int i = 0; i < count; ++i) any_stage |= n_stages[i] > 0;
        if (any_stage && !phi) fail(GFT_ERR_INVALID_ARG, "phi is NULL");
        std::vector<gft_plan_t> tmp(count, nullptr);
        create_plans(count, n, L, n_stages, phi, flags, tmp.data());
        std::copy(tmp.begin(), tmp.end(), out);
    });
}

gft_status gft_plan_create_bipartite(int32_t n, const double* L, const int32_t* side, uint32_t flags,
                                     gft_plan_t* out) {
    return guard([&] {
        if (!out) fail(GFT_ERR_INVALID_ARG, "out is NULL");
        check_create_args(n, L, 0, nullptr, flags);
        if (flags & (GFT_SPLIT_COMPONENTS | GFT_SEARCH_STAGES))
            fail(GFT_ERR_INVALID_ARG, "GFT_SPLIT_COMPONENTS and GFT_SEARCH_STAGES do not apply to bipartite plans");
        std::unique_ptr<gft_plan_s> p(new gft_plan_s);
        p->n = n;
        p->flags = flags;
        Leaf J;
        std::vector<double> Ln;
        if (flags & GFT_NORMALIZED) Ln = normalized_copy(n, L);
        analyze_bipartite(*p, Ln.empty() ? L : Ln.data(), side, J);
        if (!(flags & GFT_ANALYZE_ONLY)) {
            GFT_CUDA(cudaGetDevice(&p->device));
            cudaStream_t st = nullptr;
            GFT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            try {
                jacobi_leaf_ptrs({&J}, st);
            } catch (...) {
                cudaStreamDestroy(st);
                throw;
            }
            GFT_CUDA(cudaStreamDestroy(st));
            finish_bipartite(*p, J);
            finalize_host(*p);
            upload_plan(*p);
            jit_build(*p);
            wide_build(*p);
            GFT_CUDA(cudaDeviceSynchronize());
        }
        *out = p.release();
    });
}

gft_status gft_find_involution(int32_t n, const double* L, const int32_t* classes, int64_t max_steps, int32_t* phi,
                               int32_t* pairs) {
    return guard([&] {
        if (n < 1 || n > 4096) fail(GFT_ERR_INVALID_ARG, "n must be in [1, 4096]");
        if (!L || !phi) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        check_symmetric_finite(n, L);
        std::vector<int> out(n);
        const int p = find_involution(n, L, classes, max_steps > 0 ? max_steps : 1000000, 0.0, out.data());
        std::copy(out.begin(), out.end(), phi);
        if (pairs) *pairs = p;
    });
}

gft_status gft_search_stages(int32_t n, const double* L, int32_t max_stages, int64_t max_steps, int32_t* phis,
                             int32_t* n_stages) {
    return guard([&] {
        if (n < 1 || n > 4096) fail(GFT_ERR_INVALID_ARG, "n must be in [1, 4096]");
        if (!L || !phis || !n_stages) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        if (max_stages < 0 || max_stages > 16) fail(GFT_ERR_INVALID_ARG, "max_stages must be in [0, 16]");
        check_symmetric_finite(n, L);
        std::vector<int> out;
        const int s = search_stages(n, L, max_stages, max_steps > 0 ? max_steps : 1000000, out);
        std::copy(out.begin(), out.end(), phis);
        *n_stages = s;
    });
}

gft_status gft_plan_destroy(gft_plan_t plan) {
    return guard([&] { delete plan; });
}

gft_status gft_plan_get_info(gft_plan_t p, gft_plan_info_t* info) {
    return guard([&] {
        check_plan(p);
        if (!info) fail(GFT_ERR_INVALID_ARG, "info is NULL");
        gft_plan_info_t r{};
        r.n = p->n;
        r.n_stages = p->n_stages;
        r.n_leaves = (int32_t)p->leaves.size();
        for (auto& s : p->stages) r.n_pairs += (int32_t)s.size();
        for (auto& lf : p->leaves) {
            const int64_t m = lf.m();
            r.max_leaf = std::max<int32_t>(r.max_leaf, (int32_t)m);
            r.fast_mults += m * m;
            r.fast_adds += m * (m - 1);
            r.jacobi_sweeps = std::max(r.jacobi_sweeps, lf.sweeps);
        }
        r.right_pairs = (int32_t)p->rpairs.size();
        r.fast_adds += 2 * (int64_t)(r.n_pairs + r.right_pairs);
        r.has_device = p->has_device ? 1 : 0;
        r.flags = p->flags;
        jit_info(*p, &r.jit, &r.tile_signals, &r.threads);
        r.wide = (!r.jit && wide_ready(*p, false)) ? 1 : 0;
        *info = r;
    });
}

gft_status gft_plan_get_stage_pairs(gft_plan_t p, int32_t stage, int32_t* pairs, int32_t* count) {
    return guard([&] {
        check_plan(p);
        if (!count) fail(GFT_ERR_INVALID_ARG, "count is NULL");
        if (stage < 0 || stage >= p->n_stages) fail(GFT_ERR_INVALID_ARG, "stage out of range");
        const auto& st = p->stages[stage];
        if (!pairs) {
            *count = (int32_t)st.size();
            return;
        }
        if (*count < (int32_t)st.size()) fail(GFT_ERR_INVALID_ARG, "pairs capacity too small");
        for (size_t k = 0; k < st.size(); ++k) {
            pairs[2 * k] = st[k].first;
            pairs[2 * k + 1] = st[k].second;
        }
        *count = (int32_t)st.size();
    });
}

gft_status gft_plan_get_leaves(gft_plan_t p, int32_t* sizes, int32_t* labels) {
    return guard([&] {
        check_plan(p);
        if (!sizes || !labels) fail(GFT_ERR_INVALID_ARG, "NULL output");
        size_t o = 0;
        for (size_t k = 0; k < p->leaves.size(); ++k) {
            sizes[k] = p->leaves[k].m();
            for (int v : p->leaves[k].labels) labels[o++] = v;
        }
    });
}

gft_status gft_plan_get_leaf_laplacian(gft_plan_t p, int32_t leaf, double* Lk) {
    return guard([&] {
        check_plan(p);
        if (!Lk) fail(GFT_ERR_INVALID_ARG, "NULL output");
        if (leaf < 0 || leaf >= (int32_t)p->leaves.size()) fail(GFT_ERR_INVALID_ARG, "leaf out of range");
        if (p->right) fail(GFT_ERR_UNSUPPORTED, "the sub-transforms of a bipartite plan have no leaf Laplacian");
        const auto& v = p->leaves[leaf].L;
        std::memcpy(Lk, v.data(), v.size() * sizeof(double));
    });
}

gft_status gft_plan_get_output_map(gft_plan_t p, int32_t* out_pos) {
    return guard([&] {
        check_device_plan(p);
        if (!out_pos) fail(GFT_ERR_INVALID_ARG, "NULL output");
        for (size_t i = 0; i < p->out_pos.size(); ++i) out_pos[i] = p->out_pos[i];
    });
}

gft_status gft_plan_eigenvalues(gft_plan_t p, double* lambda) {
    return guard([&] {
        check_device_plan(p);
        if (!lambda) fail(GFT_ERR_INVALID_ARG, "NULL output");
        std::memcpy(lambda, p->lam_out.data(), sizeof(double) * p->n);
    });
}

gft_status gft_plan_basis(gft_plan_t p, double* U) {
    return guard([&] {
        check_device_plan(p);
        if (!U) fail(GFT_ERR_INVALID_ARG, "NULL output");
        compute_basis(*p, U);
    });
}

// CUDA-core transform: the plan-specialised kernel if the plan has one, the
// wide-leaf kernel for leaves over 32 nodes, else the table-driven kernel.
static void core_f32(gft_plan_s& p, const float* x, float* y, int64_t batch, bool inverse, cudaStream_t st) {
    if (jit_launch(p, false, x, y, batch, inverse, st)) return;
    if (wide_ready(p, false)) return launch_wide_f32(p, x, y, batch, inverse, st);
    launch_apply_f32(apply_args(p, false), x, y, batch, inverse, st);
}
static void core_f64(gft_plan_s& p, const double* x, double* y, int64_t batch, bool inverse, cudaStream_t st) {
    if (jit_launch(p, true, x, y, batch, inverse, st)) return;
    if (wide_ready(p, true)) return launch_wide_f64(p, x, y, batch, inverse, st);
    launch_apply_f64(apply_args(p, true), x, y, batch, inverse, st);
}

static void check_precision(gft_plan_s* p, uint32_t precision) {
    if (precision > GFT_PREC_FP16X3) fail(GFT_ERR_INVALID_ARG, "unknown precision");
    (void)p;
}

gft_status gft_plan_forward(gft_plan_t p, const float* x, float* y, int64_t batch, gft_stream_t stream,
                            uint32_t precision) {
    return guard([&] {
        check_device_plan(p);
        check_io(x, y, batch);
        check_precision(p, precision);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        p->last_stream = st;
        if (batch == 0) return;
        if (precision == GFT_PREC_FP32) {
            core_f32(*p, x, y, batch, false, st);
        } else {
            launch_tc(*p, x, y, batch, false, st, precision);
        }
    });
}

gft_status gft_plan_inverse(gft_plan_t p, const float* y, float* x, int64_t batch, gft_stream_t stream,
                            uint32_t precision) {
    return guard([&] {
        check_device_plan(p);
        check_io(y, x, batch);
        check_precision(p, precision);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        p->last_stream = st;
        if (batch == 0) return;
        if (precision == GFT_PREC_FP32) {
            core_f32(*p, y, x, batch, true, st);
        } else {
            launch_tc(*p, y, x, batch, true, st, precision);
        }
    });
}

gft_status gft_plan_forward_f64(gft_plan_t p, const double* x, double* y, int64_t batch, gft_stream_t stream) {
    return guard([&] {
        check_device_plan(p);
        check_io(x, y, batch);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        p->last_stream = st;
        core_f64(*p, x, y, batch, false, st);
    });
}

gft_status gft_plan_inverse_f64(gft_plan_t p, const double* y, double* x, int64_t batch, gft_stream_t stream) {
    return guard([&] {
        check_device_plan(p);
        check_io(y, x, batch);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        p->last_stream = st;
        core_f64(*p, y, x, batch, true, st);
    });
}

gft_status gft_plan_forward_host(gft_plan_t p, const float* x_host, float* y_host, int64_t batch,
                                 uint32_t precision) {
    return guard([&] {
        check_device_plan(p);
        if (batch < 0) fail(GFT_ERR_INVALID_ARG, "batch < 0");
        if (batch == 0) return;
        if (!x_host || !y_host) fail(GFT_ERR_INVALID_ARG, "NULL host pointer");
        check_precision(p, precision);
        const int n = p->n;
        constexpr int NB = gft_plan_s::kHostStreams;
        for (int b = 0; b < NB; ++b)
            if (!p->host_streams[b]) GFT_CUDA(cudaStreamCreateWithFlags(&p->host_streams[b], cudaStreamNonBlocking));
        // Pinned, device-mapped host buffers: the transform kernel reads and
        // writes host memory directly (no copy engines, no staging).
        if (precision == GFT_PREC_FP32) {
            cudaPointerAttributes ax{}, ay{};
            const bool qx = cudaPointerGetAttributes(&ax, x_host) == cudaSuccess;
            const bool qy = cudaPointerGetAttributes(&ay, y_host) == cudaSuccess;
            cudaGetLastError();
            if (qx && qy && ax.type == cudaMemoryTypeHost && ay.type == cudaMemoryTypeHost && ax.devicePointer &&
                ay.devicePointer && !((reinterpret_cast<uintptr_t>(ax.devicePointer) |
                                       reinterpret_cast<uintptr_t>(ay.devicePointer)) & 15u)) {
                const float* xd = static_cast<const float*>(ax.devicePointer);
                float* yd = static_cast<float*>(ay.devicePointer);
                cudaStream_t st = p->host_streams[1];
                if (!jit_launch_plain(*p, xd, yd, batch, st)) core_f32(*p, xd, yd, batch, false, st);
                GFT_CUDA(cudaStreamSynchronize(st));
                p->last_stream = nullptr;
                return;
            }
        }
        // Otherwise chunks (a quarter of the batch, 16..64 MB) flow through a
        // ring of NB device buffer pairs.  Uploads, transforms and downloads
        // run on three streams chained by events, so the host-to-device copy
        // of a chunk overlaps the device-to-host copy of an earlier one.
        const int64_t row_bytes = (int64_t)n * sizeof(float);
        int64_t chunk = std::min<int64_t>(std::max<int64_t>((batch + 3) / 4, (16ll << 20) / row_bytes),
                                          (64ll << 20) / row_bytes);
        chunk = std::max<int64_t>(4, (chunk + 3) & ~int64_t(3));
        const size_t elems = (size_t)chunk * n;
        if (p->stage_elems < elems) {
            for (int b = 0; b < NB; ++b) {
                if (p->d_stage[b]) cudaFree(p->d_stage[b]);
                if (p->d_stage_out[b]) cudaFree(p->d_stage_out[b]);
                p->d_stage[b] = p->d_stage_out[b] = nullptr;
            }
            p->stage_elems = 0;
            for (int b = 0; b < NB; ++b) {
                GFT_CUDA(cudaMalloc(&p->d_stage[b], elems * sizeof(float)));
                GFT_CUDA(cudaMalloc(&p->d_stage_out[b], elems * sizeof(float)));
            }
            p->stage_elems = elems;
        }
        for (int b = 0; b < NB; ++b) {
            for (cudaEvent_t* e : {&p->ev_up[b], &p->ev_k[b], &p->ev_down[b]})
                if (!*e) GFT_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        }
        cudaStream_t s_up = p->host_streams[0], s_k = p->host_streams[1], s_down = p->host_streams[2];
        int64_t done = 0;
        for (int64_t i = 0; done < batch; ++i) {
            const int b = (int)(i % NB);
            const int64_t rows = std::min(chunk, batch - done);
            const size_t bytes = (size_t)rows * n * sizeof(float);
            if (i >= NB) GFT_CUDA(cudaStreamWaitEvent(s_up, p->ev_k[b], 0));      // input buffer free
            GFT_CUDA(cudaMemcpyAsync(p->d_stage[b], x_host + (size_t)done * n, bytes, cudaMemcpyHostToDevice, s_up));
            GFT_CUDA(cudaEventRecord(p->ev_up[b], s_up));
            GFT_CUDA(cudaStreamWaitEvent(s_k, p->ev_up[b], 0));
            if (i >= NB) GFT_CUDA(cudaStreamWaitEvent(s_k, p->ev_down[b], 0));   // output buffer free
            if (precision == GFT_PREC_FP32) {
                core_f32(*p, p->d_stage[b], p->d_stage_out[b], rows, false, s_k);
            } else {
                launch_tc(*p, p->d_stage[b], p->d_stage_out[b], rows, false, s_k, precision);
            }
            GFT_CUDA(cudaEventRecord(p->ev_k[b], s_k));
            GFT_CUDA(cudaStreamWaitEvent(s_down, p->ev_k[b], 0));
            GFT_CUDA(cudaMemcpyAsync(y_host + (size_t)done * n, p->d_stage_out[b], bytes, cudaMemcpyDeviceToHost, s_down));
            GFT_CUDA(cudaEventRecord(p->ev_down[b], s_down));
            done += rows;
        }
        for (int b = 0; b < NB; ++b) GFT_CUDA(cudaStreamSynchronize(p->host_streams[b]));
        p->last_stream = nullptr;
    });
}

gft_status gft_plan_kernel_source(gft_plan_t p, int32_t f64, char* buf, int64_t* len) {
    return guard([&] {
        check_device_plan(p);
        if (!len) fail(GFT_ERR_INVALID_ARG, "len is NULL");
        if (!jit_eligible(*p)) fail(GFT_ERR_UNSUPPORTED, "no plan-specialised kernel for this plan");
        const std::string s = jit_source(*p, f64 != 0);
        if (!buf) {
            *len = (int64_t)s.size() + 1;
            return;
        }
        if (*len < (int64_t)s.size() + 1) fail(GFT_ERR_INVALID_ARG, "buffer too small");
        std::memcpy(buf, s.c_str(), s.size() + 1);
        *len = (int64_t)s.size() + 1;
    });
}

gft_status gft_device_error(gft_plan_t p, int32_t* code) {
    return guard([&] {
        check_device_plan(p);
        if (!code) fail(GFT_ERR_INVALID_ARG, "code is NULL");
        GFT_CUDA(cudaStreamSynchronize(p->last_stream));
        int v = 0;
        GFT_CUDA(cudaMemcpy(&v, p->dev.d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (v) GFT_CUDA(cudaMemset(p->dev.d_err, 0, sizeof(int)));
        *code = v;
    });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// approximate GFT (approx.cpp, approx.cu)
// ---------------------------------------------------------------------------
extern "C" {

gft_status gft_approx_create(int32_t n, const double* L, int32_t n_stages, const int32_t* phi, int32_t n_layers,
                             uint32_t flags, gft_approx_t* out) {
    return guard([&] {
        if (!out) fail(GFT_ERR_INVALID_ARG, "out is NULL");
        if (n < 1 || n > 1024) fail(GFT_ERR_INVALID_ARG, "n must be in [1, 1024]");
        if (!L) fail(GFT_ERR_INVALID_ARG, "L is NULL");
        if (n_stages < 0 || n_stages > 16) fail(GFT_ERR_INVALID_ARG, "n_stages must be in [0, 16]");
        if (n_stages > 0 && !phi) fail(GFT_ERR_INVALID_ARG, "phi is NULL");
        if (n_layers < 0 || n_layers > 4096) fail(GFT_ERR_INVALID_ARG, "n_layers must be in [0, 4096]");
        if (flags & ~(GFT_SPLIT_COMPONENTS | GFT_ANALYZE_ONLY)) fail(GFT_ERR_INVALID_ARG, "unknown flag");
        std::unique_ptr<gft_approx_s> a(new gft_approx_s);
        a->n = n;
        approx_build(*a, L, n_stages, phi, n_layers, flags);
        if (!(flags & GFT_ANALYZE_ONLY)) approx_upload(*a);
        *out = a.release();
    });
}

gft_status gft_approx_destroy(gft_approx_t a) {
    return guard([&] { delete a; });
}

gft_status gft_approx_get_info(gft_approx_t a, gft_approx_info_t* info) {
    return guard([&] {
        if (!a || !info) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        gft_approx_info_t r{};
        r.n = a->n;
        r.n_haar_layers = a->n_haar_layers;
        r.n_layers = (int32_t)a->layer_off.size() - 1;
        r.n_units = (int32_t)(a->pairs.size() / 2);
        r.has_device = a->has_device ? 1 : 0;
        r.tile_signals = a->ts;
        const int64_t haar = a->layer_off[a->n_haar_layers];
        r.mults = 2 * haar + 4 * (int64_t)(r.n_units - haar);
        r.adds = 2 * (int64_t)r.n_units;
        *info = r;
    });
}

gft_status gft_approx_get_units(gft_approx_t a, int32_t* layer_off, int32_t* pairs, double* coef, int32_t* perm) {
    return guard([&] {
        if (!a || !layer_off || !pairs || !coef || !perm) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        std::copy(a->layer_off.begin(), a->layer_off.end(), layer_off);
        std::copy(a->pairs.begin(), a->pairs.end(), pairs);
        std::copy(a->coef.begin(), a->coef.end(), coef);
        std::copy(a->perm.begin(), a->perm.end(), perm);
    });
}

gft_status gft_approx_eigenvalues(gft_approx_t a, double* lambda) {
    return guard([&] {
        if (!a || !lambda) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        std::copy(a->lam.begin(), a->lam.end(), lambda);
    });
}

gft_status gft_approx_basis(gft_approx_t a, double* U) {
    return guard([&] {
        if (!a || !U) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        const int n = a->n;
        // row i of the transform of e_i is row i of U_hat (node order), then the permutation
        std::vector<double> W((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i) W[(size_t)i * n + i] = 1.0;
        const size_t units = a->pairs.size() / 2;
        for (size_t u = 0; u < units; ++u) {
            const int p = a->pairs[2 * u], q = a->pairs[2 * u + 1];
            const double* m = &a->coef[4 * u];
            for (int i = 0; i < n; ++i) {
                const double xp = W[(size_t)i * n + p], xq = W[(size_t)i * n + q];
                W[(size_t)i * n + p] = m[0] * xp + m[1] * xq;
                W[(size_t)i * n + q] = m[2] * xp + m[3] * xq;
            }
        }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) U[(size_t)i * n + j] = W[(size_t)i * n + a->perm[j]];
    });
}

gft_status gft_approx_forward(gft_approx_t a, const float* x, float* y, int64_t batch, gft_stream_t stream) {
    return guard([&] {
        if (!a) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        if (!a->has_device) fail(GFT_ERR_NO_DEVICE, "approximate GFT was created with GFT_ANALYZE_ONLY");
        check_io(x, y, batch);
        if (batch > 0 && x == y) fail(GFT_ERR_INVALID_ARG, "x and y must differ");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        a->last_stream = st;
        launch_approx(*a, x, y, batch, st);
    });
}

}  // extern "C"

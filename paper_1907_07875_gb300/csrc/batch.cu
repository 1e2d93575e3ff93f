// Mixed batches: many plans (graphs of different sizes and structures),
// each with its own batch of signals, transformed forward by ONE persistent
// kernel launch that is captured in a CUDA graph and replayed.
//
// Work list: plan p contributes ceil(batch_p / TS_p) items, one per tile of
// TS_p = RS_p * 128 signals.  Plans are ordered by decreasing cost per item
// so the long items start first.  Every CTA repeatedly takes the next item
// from a device counter (atomicAdd), finds its plan by binary search over
// the plans' first item indices, reloads the plan's program (stage pairs,
// node lists, leaf matrices) into shared memory only when the plan changes,
// and runs the same table-driven tile code as the single-plan kernel
// (apply_core.cuh): cp.async tile load, in-place stages and leaf products,
// permuted coalesced store.
//
// Autotuner: at creation, every plan is timed alone in this kernel with each
// admissible RS_p (signals per thread: 1, 2 or 4, limited by the plan's leaf
// widths) on a scratch batch, and the fastest tile shape is kept.
//
// The counter lives in device memory owned by the batch and is reset by a
// memset node at the start of every replay.  Changing the signal pointers
// only rewrites the per-plan descriptors in device memory; the captured graph
// is reused.
#include <algorithm>
#include <map>
#include <memory>
#include <numeric>
#include <vector>

#include "apply_core.cuh"

namespace gft {
using namespace core;
namespace {

constexpr int kBatchThreads = 128;
constexpr int kTcMinLeaf = 64;   // leaves this wide go to the tensor cores in a tensor-core batch
constexpr int kBatchSmemLimit = 232448;

struct BatchPlanDev {
    const int* ints;
    const float* mats;
    const float* x;
    float* y;
    long long batch;
    long long item0;      // first item index of this plan
    int n, np, n_pairs, n_leaves, ints_count, n_pre_pairs;
    int off_labels, off_outpos, off_src, off_desc;
    int mats_smem, rs, ts;
    float inv_n;
};

__global__ void __launch_bounds__(kBatchThreads) gft_batch_kernel(const BatchPlanDev* __restrict__ plans, int n_plans,
                                                                 long long total_items,
                                                                 unsigned long long* counter, int mats_cap,
                                                                 int ints_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* mats = reinterpret_cast<float*>(smem_raw);
    int* ints = reinterpret_cast<int*>(smem_raw + sizeof(float) * mats_cap);
    float* tile_buf = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(ints) + sizeof(int) * ints_cap);
    __shared__ long long s_item;
    __shared__ int s_plan;
    const int tid = threadIdx.x;
    int loaded = -1;
    while (true) {
        if (tid == 0) {
            const long long it = (long long)atomicAdd(counter, 1ull);
            int p = 0;
            if (it < total_items) {
                int lo = 0, hi = n_plans - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (plans[mid].item0 <= it) lo = mid;
                    else hi = mid - 1;
                }
                p = lo;
            }
            s_item = it;
            s_plan = p;
        }
        __syncthreads();
        const long long it = s_item;
        const int p = s_plan;
        if (it >= total_items) break;
        const BatchPlanDev D = plans[p];
        KArgs a{};
        a.ints = D.ints;
        a.mats = D.mats;
        a.x = D.x;
        a.y = D.y;
        a.batch = D.batch;
        a.n = D.n;
        a.np = D.np;
        a.n_pairs = D.n_pairs;
        a.n_pre_pairs = D.n_pre_pairs;
        a.n_leaves = D.n_leaves;
        a.ints_count = D.ints_count;
        a.off_labels = D.off_labels;
        a.off_outpos = D.off_outpos;
        a.off_src = D.off_src;
        a.off_desc = D.off_desc;
        a.mats_smem = D.mats_smem;
        a.ts = D.ts;
        a.nbuf = 1;
        a.inverse = 0;
        a.inv_n = D.inv_n;
        if (p != loaded) {
            for (int i = tid; i < D.ints_count; i += kBatchThreads) ints[i] = D.ints[i];
            __syncthreads();
            const int* desc = ints + D.off_desc;
            for (int k = 0; k < D.n_leaves; ++k) {
                const int bk = desc[kLeafDesc * k + 1];
                const float* src = D.mats + desc[kLeafDesc * k + 3];
                float* dst = mats + desc[kLeafDesc * k + 4];
                for (int e = tid; e < bk * bk; e += kBatchThreads) dst[e] = src[e];
            }
            loaded = p;
        }
        const long long tile = it - D.item0;
        const int* src_slot = ints + D.off_src;
        issue_tile_load<float, kBatchThreads>(a, src_slot, tile_buf, tile);
        cp_async_commit();
        cp_async_wait0();
        __syncthreads();
        if (D.rs == 4) compute_tile<float, 4, kBatchThreads>(a, ints, mats, tile_buf);
        else if (D.rs == 2) compute_tile<float, 2, kBatchThreads>(a, ints, mats, tile_buf);
        else compute_tile<float, 1, kBatchThreads>(a, ints, mats, tile_buf);
        __syncthreads();
        store_tile<float, kBatchThreads>(a, src_slot, tile_buf, tile);
        __syncthreads();
    }
}

int rs_cap(int max_bucket) { return max_bucket <= 16 ? 4 : (max_bucket <= 32 ? 2 : 1); }

}  // namespace
}  // namespace gft

using namespace gft;

struct gft_batch_s {
    // routing of the caller's plans: 0 = table-driven batch kernel, 1 = wide-leaf
    // batch kernel, 2 = tensor-core sequence; idx = position within its group
    uint32_t precision = GFT_PREC_FP32;
    std::vector<int> kind, idx;
    std::vector<int64_t> user_batch;
    std::vector<int> table_users, wide_users, tc_users;
    std::vector<gft_plan_s*> tc_plans;
    std::vector<int64_t> tc_batches;
    void* wide = nullptr;                  // wide-leaf group (wide.cu)
    void* tcb = nullptr;                   // tensor-core group (tc.cu)
    cudaStream_t side[2] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {};
    // table-driven group
    std::vector<gft_plan_s*> plans;        // table-driven group, group order
    std::vector<int64_t> batches;
    std::vector<int> order;                // descriptor slot -> user index
    std::vector<int> rs;                   // per user index
    std::vector<BatchPlanDev> desc;        // descriptor slot order
    BatchPlanDev* d_desc = nullptr;
    unsigned long long* d_counter = nullptr;
    long long total_items = 0;
    int mats_cap = 0, ints_cap = 0;
    size_t smem = 0;
    int grid = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> last_x, last_y;
    ~gft_batch_s() {
        if (wide) gft::wide_batch_free(wide);
        if (tcb) gft::tc_batch_free(tcb);
        for (auto& st : side)
            if (st) cudaStreamDestroy(st);
        if (ev_fork) cudaEventDestroy(ev_fork);
        for (auto& e : ev_join)
            if (e) cudaEventDestroy(e);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (d_desc) cudaFree(d_desc);
        if (d_counter) cudaFree(d_counter);
    }
};

namespace gft {
namespace {

BatchPlanDev make_desc(const gft_plan_s& p, int rs, int64_t batch) {
    BatchPlanDev d{};
    d.ints = p.dev.d_ints;
    d.mats = p.dev.d_mats32;
    d.batch = batch;
    d.n = p.n;
    d.np = p.n | 1;
    d.n_pairs = p.dev.n_pairs;
    d.n_pre_pairs = p.dev.n_pre_pairs;
    d.n_leaves = p.dev.n_leaves;
    d.ints_count = p.dev.ints_count;
    d.off_labels = 2 * p.dev.n_pairs + p.dev.n_stages + 1;
    d.off_outpos = d.off_labels + p.n;
    d.off_src = d.off_outpos + p.n;
    d.off_desc = d.off_src + p.n;
    d.mats_smem = p.dev.mats_smem;
    d.rs = rs;
    d.ts = rs * kBatchThreads;
    d.inv_n = 1.0f / (float)p.n;
    return d;
}

// lays out items and sizes shared memory for the current rs choices
void layout(gft_batch_s& b) {
    const int k = (int)b.plans.size();
    std::vector<double> cost(k);
    for (int i = 0; i < k; ++i) {
        double fl = 0;
        for (auto& lf : b.plans[i]->leaves) fl += (double)lf.m() * lf.m();
        cost[i] = (fl + 8.0 * b.plans[i]->n) * b.rs[i];
    }
    b.order.resize(k);
    std::iota(b.order.begin(), b.order.end(), 0);
    std::stable_sort(b.order.begin(), b.order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    b.desc.clear();
    b.total_items = 0;
    b.mats_cap = 0;
    b.ints_cap = 0;
    size_t tile_cap = 0;
    for (int slot = 0; slot < k; ++slot) {
        const int i = b.order[slot];
        BatchPlanDev d = make_desc(*b.plans[i], b.rs[i], b.batches[i]);
        d.item0 = b.total_items;
        b.total_items += (b.batches[i] + d.ts - 1) / d.ts;
        b.desc.push_back(d);
        b.mats_cap = std::max(b.mats_cap, d.mats_smem);
        b.ints_cap = std::max(b.ints_cap, (d.ints_count + 3) & ~3);
        tile_cap = std::max(tile_cap, (size_t)d.ts * d.np);
    }
    b.mats_cap = (b.mats_cap + 3) & ~3;
    b.smem = sizeof(float) * (size_t)b.mats_cap + sizeof(int) * (size_t)b.ints_cap + sizeof(float) * tile_cap;
    if (b.smem > (size_t)kBatchSmemLimit) fail(GFT_ERR_UNSUPPORTED, "mixed batch needs too much shared memory per CTA");
}

void upload_desc(gft_batch_s& b, const float* const* x, float* const* y, cudaStream_t st) {
    for (size_t slot = 0; slot < b.desc.size(); ++slot) {
        const int i = b.order[slot];
        b.desc[slot].x = x ? x[i] : nullptr;
        b.desc[slot].y = y ? y[i] : nullptr;
    }
    GFT_CUDA(cudaMemcpyAsync(b.d_desc, b.desc.data(), sizeof(BatchPlanDev) * b.desc.size(), cudaMemcpyHostToDevice, st));
}

void launch_batch(gft_batch_s& b, cudaStream_t st) {
    GFT_CUDA(cudaMemsetAsync(b.d_counter, 0, sizeof(unsigned long long), st));
    if (b.total_items == 0) return;
    gft_batch_kernel<<<b.grid, kBatchThreads, b.smem, st>>>(b.d_desc, (int)b.desc.size(), b.total_items, b.d_counter,
                                                          b.mats_cap, b.ints_cap);
    GFT_CUDA(cudaGetLastError());
}

void configure(gft_batch_s& b) {
    GFT_CUDA(cudaFuncSetAttribute(gft_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem));
    int per_sm = 0;
    GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gft_batch_kernel, kBatchThreads, b.smem));
    if (per_sm < 1) fail(GFT_ERR_UNSUPPORTED, "mixed-batch kernel does not fit on an SM");
    b.grid = per_sm * sm_count();
}

// time plan i alone with each admissible RS; keep the fastest
void autotune(gft_batch_s& b) {
    const int k = (int)b.plans.size();
    b.rs.assign(k, 1);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* dx = nullptr;
    float* dy = nullptr;
    size_t cap = 0;
    gft_batch_s probe;
    auto cleanup = [&] {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        if (dx) cudaFree(dx);
        if (dy) cudaFree(dy);
        probe.d_desc = nullptr;
        probe.d_counter = nullptr;
    };
    try {
        GFT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        GFT_CUDA(cudaEventCreate(&e0));
        GFT_CUDA(cudaEventCreate(&e1));
        probe.d_desc = b.d_desc;
        probe.d_counter = b.d_counter;
        for (int i = 0; i < k; ++i) {
            const int n = b.plans[i]->n;
            const int64_t tb = std::max<int64_t>(1, std::min<int64_t>(b.batches[i], (int64_t)(8 << 20) / n));
            if (cap < (size_t)tb * n) {
                if (dx) cudaFree(dx);
                if (dy) cudaFree(dy);
                dx = dy = nullptr;
                cap = (size_t)tb * n;
                GFT_CUDA(cudaMalloc(&dx, cap * sizeof(float)));
                GFT_CUDA(cudaMalloc(&dy, cap * sizeof(float)));
                GFT_CUDA(cudaMemset(dx, 0, cap * sizeof(float)));
            }
            const int rmax = rs_cap(b.plans[i]->dev.max_bucket);
            float best = 0.f;
            int best_rs = 1;
            for (int rs = 1; rs <= rmax; rs *= 2) {
                probe.plans = {b.plans[i]};
                probe.batches = {tb};
                probe.rs = {rs};
                layout(probe);
                configure(probe);
                upload_desc(probe, (const float* const*)&dx, &dy, st);
                launch_batch(probe, st);
                GFT_CUDA(cudaEventRecord(e0, st));
                for (int r = 0; r < 3; ++r) launch_batch(probe, st);
                GFT_CUDA(cudaEventRecord(e1, st));
                GFT_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                GFT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (rs == 1 || ms < best) {
                    best = ms;
                    best_rs = rs;
                }
            }
            b.rs[i] = best_rs;
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

template <class F> gft_status guard_b(F&& f) {
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

}  // namespace
}  // namespace gft

extern "C" {

gft_status gft_batch_create(int32_t n_plans, const gft_plan_t* plans, const int64_t* batches, uint32_t flags,
                            gft_batch_t* out) {
    return guard_b([&] {
        if (!out || !plans || !batches || n_plans < 1) fail(GFT_ERR_INVALID_ARG, "bad arguments");
        if (flags > GFT_PREC_FP16X3) fail(GFT_ERR_INVALID_ARG, "unknown flag");
        std::unique_ptr<gft_batch_s> b(new gft_batch_s);
        b->precision = flags;
        std::vector<gft_plan_s*> wide_plans;
        std::vector<int64_t> wide_batches;
        for (int i = 0; i < n_plans; ++i) {
            gft_plan_s* p = plans[i];
            if (!p) fail(GFT_ERR_INVALID_ARG, "NULL plan");
            if (!p->has_device) fail(GFT_ERR_NO_DEVICE, "plan without device data");
            if (batches[i] < 0) fail(GFT_ERR_INVALID_ARG, "negative batch");
            int max_leaf = 0;
            for (auto& lf : p->leaves) max_leaf = std::max(max_leaf, lf.m());
            int kind;
            if (b->precision != GFT_PREC_FP32 && tc_eligible(*p) && max_leaf >= kTcMinLeaf) kind = 2;
            else if (p->dev.max_bucket != 0 && !(wide_configured(*p) && wide_ready(*p, false))) kind = 0;
            else if (wide_configured(*p)) kind = 1;
            else fail(GFT_ERR_UNSUPPORTED, "plan " + std::to_string(i) + " has a leaf wider than 512 nodes");
            b->kind.push_back(kind);
            b->user_batch.push_back(batches[i]);
            if (kind == 0) {
                b->idx.push_back((int)b->plans.size());
                b->table_users.push_back(i);
                b->plans.push_back(p);
                b->batches.push_back(batches[i]);
            } else if (kind == 1) {
                b->idx.push_back((int)wide_plans.size());
                b->wide_users.push_back(i);
                wide_plans.push_back(p);
                wide_batches.push_back(batches[i]);
            } else {
                b->idx.push_back((int)b->tc_plans.size());
                b->tc_users.push_back(i);
                b->tc_plans.push_back(p);
                b->tc_batches.push_back(batches[i]);
            }
        }
        GFT_CUDA(cudaMalloc(&b->d_desc, sizeof(BatchPlanDev) * std::max<size_t>(1, b->plans.size())));
        GFT_CUDA(cudaMalloc(&b->d_counter, sizeof(unsigned long long)));
        if (!b->plans.empty()) {
            autotune(*b);
            layout(*b);
            configure(*b);
        }
        if (!wide_plans.empty()) b->wide = wide_batch_create(wide_plans, wide_batches);
        if (!b->tc_plans.empty()) b->tcb = tc_batch_create(b->tc_plans, b->tc_batches, b->precision);
        GFT_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        for (auto& st : b->side) GFT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        GFT_CUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
        for (auto& e : b->ev_join) GFT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        *out = b.release();
    });
}

gft_status gft_batch_forward(gft_batch_t b, const float* const* x, float* const* y, gft_stream_t stream) {
    return guard_b([&] {
        if (!b || !x || !y) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        const int k = (int)b->kind.size();
        for (int i = 0; i < k; ++i) {
            if (b->user_batch[i] == 0) continue;
            if (!x[i] || !y[i]) fail(GFT_ERR_INVALID_ARG, "NULL signal pointer");
            if ((reinterpret_cast<uintptr_t>(x[i]) | reinterpret_cast<uintptr_t>(y[i])) & 15u)
                fail(GFT_ERR_MISALIGNED, "signal pointers must be 16-byte aligned");
            if (b->kind[i] == 2 && x[i] == y[i]) fail(GFT_ERR_UNSUPPORTED, "tensor-core entries do not run in place");
        }
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        const bool same = b->last_x.size() == (size_t)k &&
                          std::equal(x, x + k, b->last_x.begin()) &&
                          std::equal(y, y + k, b->last_y.begin(), [](float* a, const void* c) { return a == c; });
        if (!same) {
            // every group reads its signal pointers from device descriptors,
            // so the captured graph stays valid
            std::vector<const float*> tx, wx, cx;
            std::vector<float*> ty, wy, cy;
            for (int i : b->table_users) {
                tx.push_back(x[i]);
                ty.push_back(y[i]);
            }
            for (int i : b->wide_users) {
                wx.push_back(x[i]);
                wy.push_back(y[i]);
            }
            for (int i : b->tc_users) {
                cx.push_back(x[i]);
                cy.push_back(y[i]);
            }
            if (!b->plans.empty()) upload_desc(*b, tx.data(), ty.data(), st);
            if (b->wide) wide_batch_upload(b->wide, wx, wy, st);
            if (b->tcb) tc_batch_upload(b->tcb, cx, cy, st);
            b->last_x.assign(x, x + k);
            b->last_y.assign(y, y + k);
        }
        if (!b->exec) {
            // capture once on a private stream; the groups run on forked
            // streams and join before the graph ends
            GFT_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
            try {
                cudaStream_t cs = b->cap_stream;
                GFT_CUDA(cudaEventRecord(b->ev_fork, cs));
                bool used[2] = {false, false};
                auto fork = [&](int s) {
                    if (!used[s]) GFT_CUDA(cudaStreamWaitEvent(b->side[s], b->ev_fork, 0));
                    used[s] = true;
                    return b->side[s];
                };
                if (b->wide) wide_batch_launch(b->wide, fork(0));
                if (b->tcb) tc_batch_launch(b->tcb, fork(1));
                if (!b->plans.empty()) launch_batch(*b, cs);
                for (int s = 0; s < 2; ++s)
                    if (used[s]) {
                        GFT_CUDA(cudaEventRecord(b->ev_join[s], b->side[s]));
                        GFT_CUDA(cudaStreamWaitEvent(cs, b->ev_join[s], 0));
                    }
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(b->cap_stream, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            GFT_CUDA(cudaStreamEndCapture(b->cap_stream, &b->graph));
            GFT_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
        }
        GFT_CUDA(cudaGraphLaunch(b->exec, st));
    });
}

gft_status gft_batch_get_tile(gft_batch_t b, int32_t i, int32_t* tile, int32_t* threads) {
    return guard_b([&] {
        if (!b || !tile || !threads) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        if (i < 0 || i >= (int32_t)b->kind.size()) fail(GFT_ERR_INVALID_ARG, "index out of range");
        *tile = 0;
        *threads = 0;
        if (b->kind[i] == 0) {
            *tile = b->rs[b->idx[i]] * kBatchThreads;
            *threads = kBatchThreads;
        }
    });
}

gft_status gft_batch_destroy(gft_batch_t b) {
    return guard_b([&] { delete b; });
}

}  // extern "C"

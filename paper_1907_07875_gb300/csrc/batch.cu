// Mixed batches: many plans (graphs of different sizes and structures),
// each with its own batch of signals, transformed forward by persistent
// kernel launches that are captured in ONE CUDA graph and replayed.
//
// Groups, in routing order: the tensor-core kernels (tc.cu, tcn.cu) for
// plans with a leaf of 64 or more nodes in a tensor-core precision; the
// plan-specialised group (jit.cpp) for small plans that many entries share;
// the node-major kernel below for the other plans of at most 256 nodes
// without right Haar units; the thread-per-signal kernel below; the
// wide-leaf kernel (wide.cu).
//
// Thread-per-signal group (plans whose leaves all fit the CUDA-core tile
// code of apply_core.cuh, at most 64 nodes):
//   * Work list: plan p contributes ceil(batch_p / TS_p) items, one per
//     tile of TS_p = RS_p * 128 signals, plans in order of decreasing cost
//     per item.  Plans are split into size classes by their padded row
//     stride (n | 1 up to 17, 33, 65, 129, 257); each class is one launch
//     whose shared tile is sized for its own largest plan, so classes of
//     small graphs keep many CTAs per SM.
//   * Static schedule: the host cuts the class's item sequence into one
//     contiguous range per CTA of roughly equal estimated cost (bytes moved
//     plus leaf FMAs plus a fixed cost per item), and records the plan slot
//     of each range's first item.  A CTA walks its range in order, so the
//     items of one plan mostly stay on one CTA and its program (stage pairs,
//     node lists, leaf matrices) is copied into shared memory only when the
//     plan changes -- no atomics and no search per item.
//   * Pipeline: two tile buffers; the cp.async copies of item i+1 (whichever
//     plan it belongs to: the copy needs only the plan's descriptor) are in
//     flight while item i runs its in-place stages and leaf products and its
//     permuted, coalesced store (the same tile code as the single-plan
//     kernel, so outputs agree bit for bit).  Classes whose tile is too large
//     for two buffers and two CTAs per SM run single-buffered.
//
// Autotuner: at creation, every plan is timed alone in this kernel with each
// admissible RS_p (signals per thread: 1, 2 or 4, limited by the plan's leaf
// widths and by a tile of at most kTileCapBytes) on a scratch batch, and the
// fastest tile shape is kept.
//
// Changing the signal pointers only rewrites the per-plan descriptors in
// device memory; the captured graph is reused.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <vector>

#include "apply_core.cuh"

namespace gft {
using namespace core;
namespace {

constexpr int kBatchThreads = 128;
constexpr int kTcMinLeaf = 64;   // leaves this wide go to the 128-signal tensor-core kernel in a tensor-core batch
constexpr int kTcnMinLeaf = 64;  // leaves this wide go to the few-signals tensor-core kernel
constexpr int64_t kTcnMaxBatch = 4096;   // graphs with at most this many signals use the few-signals kernel
constexpr int kBatchSmemLimit = 232448;
constexpr size_t kTileCapBytes = 17408;        // largest tile a plan may choose (keeps several CTAs per SM)
constexpr size_t kDoubleBufBytes = 72 * 1024;  // two tile buffers only if they fit in this
constexpr int kClassStride[] = {17, 33, 65, 129, 257};
constexpr int kClasses = 5;

struct BatchPlanDev {
    const int* ints;
    const float* mats;
    const float* x;
    float* y;
    long long batch;
    long long item0;      // first item index of this plan within its class
    int n, np, n_pairs, n_leaves, ints_count, n_pre_pairs;
    int off_labels, off_outpos, off_src, off_desc;
    int mats_smem, rs, ts;
    float inv_n;
    int n_stages;   // node-major kernel: Haar stages before the leaves
    int lg_g;       // node-major kernel: log2(ts / 4), signal groups of four per tile
    int tsp;        // node-major kernel: signal stride of a node row (ts + 4)
    const int* nm;  // node-major kernel: program image (see DevProgram)
    int nm_words, nm_cg_off, nm_n_cg;
};

__device__ __forceinline__ KArgs batch_kargs(const BatchPlanDev& D) {
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
    return a;
}

// CTA b runs items [range[b], range[b+1]) of its class; first_slot[b] is
// the plan slot of item range[b].  plans[] holds the class's plans in slot
// order with their first item indices.
__global__ void __launch_bounds__(kBatchThreads) gft_batch_kernel(const BatchPlanDev* __restrict__ plans, int n_plans,
                                                                 const long long* __restrict__ range,
                                                                 const int* __restrict__ first_slot, int mats_cap,
                                                                 int ints_cap, int tile_cap, int nbuf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* mats = reinterpret_cast<float*>(smem_raw);
    int* ints = reinterpret_cast<int*>(smem_raw + sizeof(float) * mats_cap);
    float* bufs = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(ints) + sizeof(int) * ints_cap);
    const int tid = threadIdx.x;
    const long long it0 = range[blockIdx.x], it1 = range[blockIdx.x + 1];
    if (it0 >= it1) return;
    auto slot_of = [&](int s, long long it) {
        while (s + 1 < n_plans && plans[s + 1].item0 <= it) ++s;
        return s;
    };
    int slot = slot_of(first_slot[blockIdx.x], it0);
    {
        const BatchPlanDev D0 = plans[slot];
        issue_tile_load<float, kBatchThreads>(batch_kargs(D0), nullptr, bufs, it0 - D0.item0);
    }
    cp_async_commit();
    int loaded = -1, cur = 0;
    for (long long it = it0; it < it1; ++it) {
        const BatchPlanDev D = plans[slot];
        const KArgs a = batch_kargs(D);
        float* buf = bufs + (size_t)cur * tile_cap;
        int nslot = slot;
        if (nbuf == 2) {
            // the other buffer was released by the barrier ending the last item
            if (it + 1 < it1) {
                nslot = slot_of(slot, it + 1);
                const BatchPlanDev Dn = plans[nslot];
                issue_tile_load<float, kBatchThreads>(batch_kargs(Dn), nullptr, bufs + (size_t)(cur ^ 1) * tile_cap,
                                                      it + 1 - Dn.item0);
            }
            cp_async_commit();
        }
        if (slot != loaded) {
            // the barrier ending the last item released the old program
            for (int i = tid; i < D.ints_count; i += kBatchThreads) ints[i] = D.ints[i];
            __syncthreads();
            const int* desc = ints + D.off_desc;
            for (int k = 0; k < D.n_leaves; ++k) {
                const int bk = desc[kLeafDesc * k + 1];
                const float* src = D.mats + desc[kLeafDesc * k + 3];
                float* dst = mats + desc[kLeafDesc * k + 4];
                for (int e = tid; e < bk * bk; e += kBatchThreads) dst[e] = src[e];
            }
            loaded = slot;
        }
        if (nbuf == 2) cp_async_wait1();
        else cp_async_wait0();
        __syncthreads();   // tile and program visible to every thread
        if (D.rs == 4) compute_tile<float, 4, kBatchThreads>(a, ints, mats, buf);
        else if (D.rs == 2) compute_tile<float, 2, kBatchThreads>(a, ints, mats, buf);
        else compute_tile<float, 1, kBatchThreads>(a, ints, mats, buf);
        __syncthreads();
        store_tile<float, kBatchThreads>(a, ints + D.off_src, buf, it - D.item0);
        __syncthreads();   // buffer and program free
        if (nbuf == 2) {
            cur ^= 1;
        } else if (it + 1 < it1) {
            nslot = slot_of(slot, it + 1);
            const BatchPlanDev Dn = plans[nslot];
            issue_tile_load<float, kBatchThreads>(batch_kargs(Dn), nullptr, bufs, it + 1 - Dn.item0);
            cp_async_commit();
        }
        slot = nslot;
    }
    cp_async_wait0();
}

// Node-major variant of the table-driven batch kernel, for plans of at most
// kNmMaxN nodes without right Haar units (every leaf at most 64 nodes).
// An item is a tile of TS signals (a power of two, 16..1024, at most 4096
// floats per tile unless TS = 16) of one plan:
//   * the rows arrive with 16-byte cp.async copies into a row-major buffer
//     X, and so does the plan's program image (pairs, stage offsets, node
//     lists, leaf descriptors, the (leaf, output group) list) into one of
//     two program buffers when the plan changes: both are in flight for the
//     next item while this one runs; the leaf matrices are read through L1;
//   * a shared-memory pass transposes X into T[node][signal] (signal stride
//     TSP = TS + 4, so node rows stay 16-byte aligned);
//   * a Haar unit (x_i, x_j) -> (x_i + x_j, x_i - x_j) (Sec. III) works on
//     four signals with two 16-byte loads and two stores; the CTA takes one
//     stage at a time (the units of a stage touch disjoint nodes);
//   * the leaf products of every leaf run in one pass: a thread owns four
//     outputs c0..c0+3 of one leaf for four signals, reads x_r of the four
//     signals and row r of the leaf matrix with one 16-byte load each and
//     issues 16 FMAs; it writes its outputs straight to their coefficient
//     rows (ascending eigenvalue) of an output tile O, which reuses X;
//   * the store pass reads O transposed back and writes 16-byte stores.
// Each output is the same FMA chain (r ascending from zero) as in the
// thread-per-signal kernel, so the results agree bit for bit.
constexpr int kNmThreads = 256;
constexpr double kGroupMinCoeffs = 524288.0;   // plan-specialised group: coefficients of a plan over its entries
constexpr int kNmMaxN = 256;
constexpr int kNmMaxTs = 1024;      // signals per tile: a power of two, 16..1024
constexpr int kNmTileFloats = 4096;

__global__ void __launch_bounds__(kNmThreads, 4) gft_nm_kernel(const BatchPlanDev* __restrict__ plans, int n_plans,
                                                           const long long* __restrict__ range,
                                                           const int* __restrict__ first_slot, int prog_cap,
                                                           int buf_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* progs = reinterpret_cast<int*>(smem_raw);                 // two program buffers of prog_cap words
    float* xb = reinterpret_cast<float*>(progs + 2 * (size_t)prog_cap);
    float* T = xb + 2 * (size_t)buf_cap;
    const int tid = threadIdx.x;
    const long long it0 = range[blockIdx.x], it1 = range[blockIdx.x + 1];
    if (it0 >= it1) return;
    auto slot_of = [&](int s, long long it) {
        while (s + 1 < n_plans && plans[s + 1].item0 <= it) ++s;
        return s;
    };
    // 16-byte copies of the item's rows (contiguous in global memory: the
    // tile starts at a multiple of TS rows and the signal pointer is 16-byte
    // aligned), a 4-byte tail
    auto issue = [&](const BatchPlanDev& D, float* dst, long long item) {
        const long long row0 = item * D.ts;
        const int rows = (int)min((long long)D.ts, D.batch - row0);
        const int E = rows * D.n;
        const float* src = D.x + row0 * D.n;
        for (int q = tid; 4 * q + 3 < E; q += kNmThreads) cp_async16(dst + 4 * q, src + 4 * q);
        for (int e = (E & ~3) + tid; e < E; e += kNmThreads) cp_async4(dst + e, src + e);
    };
    auto issue_prog = [&](const BatchPlanDev& D, int* dst) {
        for (int q = tid; 4 * q < D.nm_words; q += kNmThreads) cp_async16(dst + 4 * q, D.nm + 4 * q);
    };
    int slot = slot_of(first_slot[blockIdx.x], it0);
    // which program image each buffer holds (or receives); the same in every thread
    const int* held0 = plans[slot].nm;
    const int* held1 = nullptr;
    int pc = 0;
    issue(plans[slot], xb, it0 - plans[slot].item0);
    issue_prog(plans[slot], progs);
    cp_async_commit();
    int cur = 0;
    for (long long it = it0; it < it1; ++it) {
        const BatchPlanDev D = plans[slot];
        float* X = xb + (size_t)cur * buf_cap;
        // the other tile and program buffers were released by the barrier
        // ending the last item
        int nslot = slot, npc = pc;
        if (it + 1 < it1) {
            nslot = slot_of(slot, it + 1);
            const BatchPlanDev& Dn = plans[nslot];
            issue(Dn, xb + (size_t)(cur ^ 1) * buf_cap, it + 1 - Dn.item0);
            if (Dn.nm != (pc ? held1 : held0)) {
                npc = pc ^ 1;
                if (Dn.nm != (npc ? held1 : held0)) {
                    issue_prog(Dn, progs + (size_t)npc * prog_cap);
                    (npc ? held1 : held0) = Dn.nm;
                }
            }
        }
        cp_async_commit();
        cp_async_wait1();   // this item's rows and program (the next item's may stay in flight)
        __syncthreads();
        const int* ints = progs + (size_t)pc * prog_cap;
        const int* cg = ints + D.nm_cg_off;
        const int* desc = ints + D.off_desc;
        const int n = D.n, tsp = D.tsp, tsp4 = D.tsp >> 2, lg = D.lg_g, gmask = (1 << D.lg_g) - 1;
        const long long row0 = (it - D.item0) * D.ts;
        const int rows = (int)min((long long)D.ts, D.batch - row0);
        const int E = rows * n;
        // X (row-major) -> T[node][signal].  n a multiple of 4: a 16-byte
        // chunk is four nodes of one signal, and (signal, node) of this
        // thread's chunk advances by a fixed step each pass
        const bool quad = (n & 3) == 0;
        const int step_s = 4 * kNmThreads / n, step_j = 4 * kNmThreads - step_s * n;
        const int s_first = row_of(4 * tid, D.inv_n), j_first = 4 * tid - s_first * n;
        if (quad) {
            int s = s_first, j = j_first;
            for (int q = tid; 4 * q < E; q += kNmThreads) {
                const float4 v = reinterpret_cast<const float4*>(X)[q];
                float* t = T + j * tsp + s;
                t[0] = v.x;
                t[tsp] = v.y;
                t[2 * tsp] = v.z;
                t[3 * tsp] = v.w;
                s += step_s;
                j += step_j;
                if (j >= n) {
                    j -= n;
                    ++s;
                }
            }
        } else {
            for (int q = tid; 4 * q < E; q += kNmThreads) {
                const int e = 4 * q;
                int s = row_of(e, D.inv_n), j = e - s * n;
                const float4 v = *reinterpret_cast<const float4*>(X + e);
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (e + i < E) T[j * tsp + s] = vv[i];
                    if (++j == n) {
                        j = 0;
                        ++s;
                    }
                }
            }
        }
        __syncthreads();
        float4* T4 = reinterpret_cast<float4*>(T);
        // Haar stages (the signals past the batch's end carry stale values
        // that are never stored)
        for (int st = 0; st < D.n_stages; ++st) {
            const int p0 = ints[2 * D.n_pairs + st], cnt = ints[2 * D.n_pairs + st + 1] - p0;
            for (int w = tid; w < (cnt << lg); w += kNmThreads) {
                const int2 ij = reinterpret_cast<const int2*>(ints)[p0 + (w >> lg)];
                const int g = w & gmask;
                const float4 a = T4[ij.x * tsp4 + g], b = T4[ij.y * tsp4 + g];
                T4[ij.x * tsp4 + g] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
                T4[ij.y * tsp4 + g] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
            }
            __syncthreads();
        }
        // leaf products into O (= X, whose rows were consumed above)
        float4* O4 = reinterpret_cast<float4*>(X);
        const int* labels = ints + D.off_labels;
        const int* outpos = ints + D.off_outpos;
        for (int w = tid; w < (D.nm_n_cg << lg); w += kNmThreads) {
            const int e = cg[w >> lg], g = w & gmask;
            const int* d = desc + kLeafDesc * (e >> 16);
            const int c0 = e & 0xFFFF, m = d[0], bk = d[1];
            const int* idx = labels + d[2];
            const float* M = D.mats + d[3] + c0;   // forward leaf matrix (L1-cached)
            float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll 4
            for (int r = 0; r < m; ++r) {
                const float4 x = T4[idx[r] * tsp4 + g];
                const float4 u = __ldg(reinterpret_cast<const float4*>(M + r * bk));
                a0.x = fmaf(x.x, u.x, a0.x); a0.y = fmaf(x.y, u.x, a0.y); a0.z = fmaf(x.z, u.x, a0.z); a0.w = fmaf(x.w, u.x, a0.w);
                a1.x = fmaf(x.x, u.y, a1.x); a1.y = fmaf(x.y, u.y, a1.y); a1.z = fmaf(x.z, u.y, a1.z); a1.w = fmaf(x.w, u.y, a1.w);
                a2.x = fmaf(x.x, u.z, a2.x); a2.y = fmaf(x.y, u.z, a2.y); a2.z = fmaf(x.z, u.z, a2.z); a2.w = fmaf(x.w, u.z, a2.w);
                a3.x = fmaf(x.x, u.w, a3.x); a3.y = fmaf(x.y, u.w, a3.y); a3.z = fmaf(x.z, u.w, a3.z); a3.w = fmaf(x.w, u.w, a3.w);
            }
            const int* op = outpos + d[2] + c0;
            O4[op[0] * tsp4 + g] = a0;
            if (c0 + 1 < m) O4[op[1] * tsp4 + g] = a1;
            if (c0 + 2 < m) O4[op[2] * tsp4 + g] = a2;
            if (c0 + 3 < m) O4[op[3] * tsp4 + g] = a3;
        }
        __syncthreads();
        // O[coefficient][signal] -> rows, 16-byte streaming stores
        const float* O = X;
        float* dst = D.y + row0 * n;
        if (quad) {
            int s = s_first, j = j_first;
            for (int q = tid; 4 * q < E; q += kNmThreads) {
                const float* o = O + j * tsp + s;
                __stcs(reinterpret_cast<float4*>(dst) + q, make_float4(o[0], o[tsp], o[2 * tsp], o[3 * tsp]));
                s += step_s;
                j += step_j;
                if (j >= n) {
                    j -= n;
                    ++s;
                }
            }
        }
        for (int q = quad ? E : tid; 4 * q < E; q += kNmThreads) {
            const int e = 4 * q;
            int s = row_of(e, D.inv_n), j = e - s * n;
            float v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                v[i] = e + i < E ? O[j * tsp + s] : 0.f;
                if (++j == n) {
                    j = 0;
                    ++s;
                }
            }
            if (e + 3 < E) {
                __stcs(reinterpret_cast<float4*>(dst + e), make_float4(v[0], v[1], v[2], v[3]));
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (e + i < E) __stcs(dst + e + i, v[i]);
            }
        }
        __syncthreads();   // X, T and the program buffer free
        cur ^= 1;
        slot = nslot;
        pc = npc;
    }
    cp_async_wait0();
}

int rs_cap(int max_bucket) { return max_bucket <= 16 ? 4 : (max_bucket <= 32 ? 2 : 1); }

// admissible RS for a plan: leaf widths and the tile cap (RS = 1 always)
bool rs_admissible(const gft_plan_s& p, int rs) {
    if (rs > rs_cap(p.dev.max_bucket)) return false;
    return rs == 1 || (size_t)rs * kBatchThreads * (size_t)(p.n | 1) * sizeof(float) <= kTileCapBytes;
}

int class_of(int np) {
    for (int c = 0; c < kClasses; ++c)
        if (np <= kClassStride[c]) return c;
    return kClasses - 1;
}

// One launch of the table-driven group: the plans of one size class.
struct BatchClass {
    std::vector<int> members;              // slot -> index into the group's plan list
    std::vector<BatchPlanDev> desc;        // slot order
    BatchPlanDev* d_desc = nullptr;
    long long* d_range = nullptr;          // grid + 1 item boundaries
    int* d_first = nullptr;                // grid plan slots
    long long total_items = 0;
    int mats_cap = 0, ints_cap = 0, tile_cap = 0, nbuf = 1;
    bool nm = false;                       // node-major kernel (tile_cap: floats per buffer)
    size_t smem = 0;
    int grid = 0;
    void release() {
        for (void** q : {(void**)&d_desc, (void**)&d_range, (void**)&d_first})
            if (*q) {
                cudaFree(*q);
                *q = nullptr;
            }
    }
};

}  // namespace
}  // namespace gft

using namespace gft;

struct gft_batch_s {
    // routing of the caller's plans: 0 = table-driven batch kernel, 1 = wide-leaf
    // batch kernel, 2 = tensor-core sequence (pack + leaf kernels, 128 signals
    // per tile), 3 = few-signals tensor-core kernels, 4 = node-major table-driven
    // kernel, 5 = plan-specialised group; idx = position within its group
    uint32_t precision = GFT_PREC_FP32;
    std::vector<int> kind, idx;
    std::vector<int64_t> user_batch;
    std::vector<int> table_users, wide_users, tc_users, tcn_users, nm_users, jg_users;
    std::vector<gft_plan_s*> jg_plans;
    std::vector<int64_t> jg_batches;
    void* jgroup = nullptr;                // plan-specialised group (jit.cpp)
    std::vector<gft_plan_s*> tc_plans, tcn_plans;
    std::vector<int64_t> tc_batches, tcn_batches;
    void* wide = nullptr;                  // wide-leaf group (wide.cu)
    void* tcb = nullptr;                   // tensor-core group (tc.cu)
    void* tcnb = nullptr;                  // few-signals tensor-core group (tcn.cu)
    // forked streams of the captured graph: 0 wide-leaf group, 1 tensor-core
    // groups
    static constexpr int kSide = 2;
    cudaStream_t side[kSide] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kSide] = {};
    // table-driven group
    std::vector<gft_plan_s*> plans;        // table-driven group, group order
    std::vector<int64_t> batches;
    std::vector<int> rs;                   // per group index
    std::vector<BatchClass> classes;       // non-empty size classes
    // node-major group
    std::vector<gft_plan_s*> nm_plans;
    std::vector<int64_t> nm_batches;
    std::vector<BatchClass> nm_classes;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> last_x, last_y;
    ~gft_batch_s() {
        if (wide) gft::wide_batch_free(wide);
        if (tcb) gft::tc_batch_free(tcb);
        if (tcnb) gft::tcn_batch_free(tcnb);
        if (jgroup) gft::jit_group_free(jgroup);
        for (auto& st : side)
            if (st) cudaStreamDestroy(st);
        if (ev_fork) cudaEventDestroy(ev_fork);
        for (auto& e : ev_join)
            if (e) cudaEventDestroy(e);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (auto& c : classes) c.release();
        for (auto& c : nm_classes) c.release();
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

// estimated cost of one item of `rows` signals (arbitrary units ~ ns on one
// SM): bytes in and out, leaf FMAs, and a fixed cost per item
double item_cost(const gft_plan_s& p, long long rows) {
    double fl = 0;
    for (auto& lf : p.leaves) fl += (double)lf.m() * lf.m();
    return (double)rows * (0.2 * p.n + 0.02 * fl + 0.02 * p.dev.n_pairs) + 1500.0;
}

// Cuts a class's item sequence (slots in order, items[sl] items each, item t
// of slot sl costing cost(sl, t)) into C.grid contiguous ranges of about
// equal cost, records the plan slot of each range's first item, and hands
// the class (with its device copies of the ranges) to `out`.
template <class F>
void finish_class(BatchClass&& C, const std::vector<long long>& items, F cost, std::vector<BatchClass>& out) {
    double total = 0.0;
    for (size_t sl = 0; sl < C.desc.size(); ++sl)
        for (long long t = 0; t < items[sl]; ++t) total += cost(sl, t);
    std::vector<long long> range(C.grid + 1, C.total_items);
    std::vector<int> first(C.grid, (int)C.desc.size() - 1);
    range[0] = 0;
    first[0] = 0;
    double acc = 0.0;
    int cta = 1;
    for (size_t sl = 0; sl < C.desc.size() && cta < C.grid; ++sl) {
        for (long long t = 0; t < items[sl] && cta < C.grid; ++t) {
            acc += cost(sl, t);
            while (cta < C.grid && acc >= total * cta / C.grid) {
                range[cta] = std::min(C.desc[sl].item0 + t + 1, C.total_items);
                first[cta] = (int)sl;
                ++cta;
            }
        }
    }
    // a range that starts at the first item of the next slot names the
    // slot it ends in; the kernel walks forward from there
    out.push_back(std::move(C));   // owned by the batch before any allocation
    BatchClass& D = out.back();
    GFT_CUDA(cudaMalloc(&D.d_desc, sizeof(BatchPlanDev) * D.desc.size()));
    GFT_CUDA(cudaMalloc(&D.d_range, sizeof(long long) * range.size()));
    GFT_CUDA(cudaMalloc(&D.d_first, sizeof(int) * first.size()));
    GFT_CUDA(cudaMemcpy(D.d_range, range.data(), sizeof(long long) * range.size(), cudaMemcpyHostToDevice));
    GFT_CUDA(cudaMemcpy(D.d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
}

// Builds every size class of the thread-per-signal kernel: slots (decreasing
// cost per item), item indices, shared-memory sizes, grid, per-CTA ranges.
void layout(gft_batch_s& b) {
    const int k = (int)b.plans.size();
    for (auto& c : b.classes) c.release();
    b.classes.clear();
    std::vector<std::vector<int>> by(kClasses);
    for (int i = 0; i < k; ++i) by[class_of(b.plans[i]->n | 1)].push_back(i);
    for (int ci = 0; ci < kClasses; ++ci) {
        if (by[ci].empty()) continue;
        BatchClass C;
        std::vector<double> cpi(k, 0.0);
        for (int i : by[ci]) cpi[i] = item_cost(*b.plans[i], (long long)b.rs[i] * kBatchThreads);
        C.members = by[ci];
        std::stable_sort(C.members.begin(), C.members.end(), [&](int x, int y) { return cpi[x] > cpi[y]; });
        size_t tile_cap = 0;
        std::vector<long long> items;
        for (int i : C.members) {
            BatchPlanDev d = make_desc(*b.plans[i], b.rs[i], b.batches[i]);
            d.item0 = C.total_items;
            items.push_back((b.batches[i] + d.ts - 1) / d.ts);
            C.total_items += items.back();
            C.desc.push_back(d);
            C.mats_cap = std::max(C.mats_cap, d.mats_smem);
            C.ints_cap = std::max(C.ints_cap, (d.ints_count + 3) & ~3);
            tile_cap = std::max(tile_cap, (size_t)d.ts * d.np);
        }
        C.mats_cap = (C.mats_cap + 3) & ~3;
        C.tile_cap = (int)((tile_cap + 3) & ~size_t(3));
        const size_t fixed = sizeof(float) * (size_t)C.mats_cap + sizeof(int) * (size_t)C.ints_cap;
        const size_t tile_bytes = sizeof(float) * (size_t)C.tile_cap;
        C.nbuf = 2 * tile_bytes <= kDoubleBufBytes && fixed + 2 * tile_bytes <= (size_t)kBatchSmemLimit ? 2 : 1;
        C.smem = fixed + C.nbuf * tile_bytes;
        if (C.smem > (size_t)kBatchSmemLimit) fail(GFT_ERR_UNSUPPORTED, "mixed batch needs too much shared memory per CTA");
        // the attribute is an upper bound shared by every batch: set it to the
        // limit once, so that no later batch can lower it under a captured launch
        GFT_CUDA(cudaFuncSetAttribute(gft_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmemLimit));
        int per_sm = 0;
        GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gft_batch_kernel, kBatchThreads, C.smem));
        if (per_sm < 1) fail(GFT_ERR_UNSUPPORTED, "mixed-batch kernel does not fit on an SM");
        C.grid = (int)std::max<long long>(1, std::min<long long>((long long)per_sm * sm_count(), C.total_items));
        const std::vector<int> mem = C.members;
        const std::vector<BatchPlanDev> ds = C.desc;
        finish_class(
            std::move(C), items,
            [&](size_t sl, long long t) {
                const int i = mem[sl];
                return t + 1 < items[sl] ? cpi[i] : item_cost(*b.plans[i], b.batches[i] - t * ds[sl].ts);
            },
            b.classes);
    }
}

// node-major kernel: plans it runs and their tile (signals, a power of two)
bool nm_eligible(const gft_plan_s& p) {
    return p.has_device && !p.right && p.dev.max_bucket != 0 && p.dev.d_nm && p.dev.n_pre_pairs == p.dev.n_pairs &&
           p.dev.n_pre_stages == p.dev.n_stages && p.n >= 1 && p.n <= kNmMaxN;
}

int nm_ts(int n) {
    int ts = kNmMaxTs;
    while (ts > 16 && (long long)ts * n > kNmTileFloats) ts >>= 1;
    return ts;
}

constexpr int kNmClasses = 5;
int nm_class_of(int n) { return n <= 16 ? 0 : (n <= 32 ? 1 : (n <= 64 ? 2 : (n <= 128 ? 3 : 4))); }

// Builds the node-major kernel's size classes (n up to 16, 32, 64, 128, 256).
void layout_nm(gft_batch_s& b) {
    const int k = (int)b.nm_plans.size();
    for (auto& c : b.nm_classes) c.release();
    b.nm_classes.clear();
    std::vector<std::vector<int>> by(kNmClasses);
    for (int i = 0; i < k; ++i) by[nm_class_of(b.nm_plans[i]->n)].push_back(i);
    for (int ci = 0; ci < kNmClasses; ++ci) {
        if (by[ci].empty()) continue;
        BatchClass C;
        std::vector<double> cpi(k, 0.0);
        for (int i : by[ci]) cpi[i] = item_cost(*b.nm_plans[i], nm_ts(b.nm_plans[i]->n));
        C.members = by[ci];
        std::stable_sort(C.members.begin(), C.members.end(), [&](int x, int y) { return cpi[x] > cpi[y]; });
        size_t buf_cap = 0;
        std::vector<long long> items;
        for (int i : C.members) {
            const gft_plan_s& p = *b.nm_plans[i];
            BatchPlanDev d = make_desc(p, 1, b.nm_batches[i]);
            d.ts = nm_ts(p.n);
            d.tsp = d.ts + 4;
            d.lg_g = 0;
            while ((1 << d.lg_g) < d.ts / 4) ++d.lg_g;
            d.n_stages = p.dev.n_pre_stages;
            d.nm = p.dev.d_nm;
            d.nm_words = p.dev.nm_words;
            d.nm_cg_off = p.dev.nm_cg_off;
            d.nm_n_cg = p.dev.nm_n_cg;
            d.item0 = C.total_items;
            items.push_back((b.nm_batches[i] + d.ts - 1) / d.ts);
            C.total_items += items.back();
            C.desc.push_back(d);
            C.ints_cap = std::max(C.ints_cap, d.nm_words);   // program image words (a multiple of 4)
            buf_cap = std::max(buf_cap, (size_t)p.n * d.tsp);
        }
        C.tile_cap = (int)((buf_cap + 3) & ~size_t(3));
        C.nm = true;
        C.smem = 2 * sizeof(int) * (size_t)C.ints_cap + 3 * sizeof(float) * (size_t)C.tile_cap;
        if (C.smem > (size_t)kBatchSmemLimit - 1024)
            fail(GFT_ERR_UNSUPPORTED, "mixed batch needs too much shared memory per CTA");
        GFT_CUDA(cudaFuncSetAttribute(gft_nm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmemLimit - 1024));
        int per_sm = 0;
        GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gft_nm_kernel, kNmThreads, C.smem));
        if (per_sm < 1) fail(GFT_ERR_UNSUPPORTED, "node-major batch kernel does not fit on an SM");
        C.grid = (int)std::max<long long>(1, std::min<long long>((long long)per_sm * sm_count(), C.total_items));
        const std::vector<int> mem = C.members;
        const std::vector<BatchPlanDev> ds = C.desc;
        finish_class(
            std::move(C), items,
            [&](size_t sl, long long t) {
                const int i = mem[sl];
                return t + 1 < items[sl] ? cpi[i] : item_cost(*b.nm_plans[i], b.nm_batches[i] - t * ds[sl].ts);
            },
            b.nm_classes);
    }
}

// x / y: pointers per group index (the caller's order within the group)
void upload_classes(std::vector<BatchClass>& classes, const float* const* x, float* const* y, cudaStream_t st) {
    for (auto& C : classes) {
        for (size_t slot = 0; slot < C.desc.size(); ++slot) {
            const int i = C.members[slot];
            C.desc[slot].x = x ? x[i] : nullptr;
            C.desc[slot].y = y ? y[i] : nullptr;
        }
        GFT_CUDA(cudaMemcpyAsync(C.d_desc, C.desc.data(), sizeof(BatchPlanDev) * C.desc.size(), cudaMemcpyHostToDevice,
                                 st));
    }
}

void upload_desc(gft_batch_s& b, const float* const* x, float* const* y, cudaStream_t st) {
    upload_classes(b.classes, x, y, st);
}

// stream_of(j): the stream of the j-th launched class
template <class F> void launch_nm(gft_batch_s& b, F stream_of) {
    int j = 0;
    for (auto& C : b.nm_classes) {
        if (C.total_items == 0) continue;
        gft_nm_kernel<<<C.grid, kNmThreads, C.smem, stream_of(j++)>>>(C.d_desc, (int)C.desc.size(), C.d_range,
                                                                      C.d_first, C.ints_cap, C.tile_cap);
        GFT_CUDA(cudaGetLastError());
    }
}

template <class F> void launch_batch(gft_batch_s& b, F stream_of) {
    int j = 0;
    for (auto& C : b.classes) {
        if (C.total_items == 0) continue;
        gft_batch_kernel<<<C.grid, kBatchThreads, C.smem, stream_of(j++)>>>(C.d_desc, (int)C.desc.size(), C.d_range, C.d_first,
                                                              C.mats_cap, C.ints_cap, C.tile_cap, C.nbuf);
        GFT_CUDA(cudaGetLastError());
    }
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
    };
    try {
        GFT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        GFT_CUDA(cudaEventCreate(&e0));
        GFT_CUDA(cudaEventCreate(&e1));
        // plans that are the same object share one measurement
        std::map<const gft_plan_s*, int> seen;
        for (int i = 0; i < k; ++i) {
            auto hit = seen.find(b.plans[i]);
            if (hit != seen.end()) {
                b.rs[i] = hit->second;
                continue;
            }
            const int n = b.plans[i]->n;
            const int64_t tb = std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(b.batches[i], 4096),
                                                                      (int64_t)(8 << 20) / n));
            if (cap < (size_t)tb * n) {
                if (dx) cudaFree(dx);
                if (dy) cudaFree(dy);
                dx = dy = nullptr;
                cap = (size_t)tb * n;
                GFT_CUDA(cudaMalloc(&dx, cap * sizeof(float)));
                GFT_CUDA(cudaMalloc(&dy, cap * sizeof(float)));
                GFT_CUDA(cudaMemset(dx, 0, cap * sizeof(float)));
            }
            float best = 0.f;
            int best_rs = 1;
            for (int rs = 1; rs <= 4; rs *= 2) {
                if (!rs_admissible(*b.plans[i], rs)) continue;
                probe.plans = {b.plans[i]};
                probe.batches = {tb};
                probe.rs = {rs};
                layout(probe);
                upload_desc(probe, (const float* const*)&dx, &dy, st);
                launch_batch(probe, [&](int) { return st; });
                GFT_CUDA(cudaEventRecord(e0, st));
                for (int r = 0; r < 3; ++r) launch_batch(probe, [&](int) { return st; });
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
            seen[b.plans[i]] = best_rs;
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
        if ((flags & ~GFT_BATCH_NO_JIT) > GFT_PREC_FP16X3) fail(GFT_ERR_INVALID_ARG, "unknown flag");
        std::unique_ptr<gft_batch_s> b(new gft_batch_s);
        b->precision = flags & ~GFT_BATCH_NO_JIT;
        const bool group_ok = !(flags & GFT_BATCH_NO_JIT);
        // coefficients per plan over its entries: the plan-specialised group
        // takes the small plans that many entries share
        std::map<const gft_plan_s*, double> coeffs;
        for (int i = 0; i < n_plans; ++i)
            if (plans[i] && batches[i] > 0) coeffs[plans[i]] += (double)batches[i] * plans[i]->n;
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
            const bool tc_prec = b->precision != GFT_PREC_FP32;
            const bool big_batch_tc = tc_prec && max_leaf >= kTcMinLeaf && tc_eligible(*p) && batches[i] > kTcnMaxBatch;
            if (tc_prec && max_leaf >= kTcnMinLeaf && !big_batch_tc && tcn_eligible(*p)) kind = 3;
            else if (tc_prec && max_leaf >= kTcMinLeaf && tc_eligible(*p)) kind = 2;
            else if (group_ok && coeffs[p] >= kGroupMinCoeffs && jit_group_eligible(*p)) kind = 5;
            else if (nm_eligible(*p)) kind = 4;
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
            } else if (kind == 5) {
                b->idx.push_back((int)b->jg_plans.size());
                b->jg_users.push_back(i);
                b->jg_plans.push_back(p);
                b->jg_batches.push_back(batches[i]);
            } else if (kind == 4) {
                b->idx.push_back((int)b->nm_plans.size());
                b->nm_users.push_back(i);
                b->nm_plans.push_back(p);
                b->nm_batches.push_back(batches[i]);
            } else if (kind == 2) {
                b->idx.push_back((int)b->tc_plans.size());
                b->tc_users.push_back(i);
                b->tc_plans.push_back(p);
                b->tc_batches.push_back(batches[i]);
            } else {
                b->idx.push_back((int)b->tcn_plans.size());
                b->tcn_users.push_back(i);
                b->tcn_plans.push_back(p);
                b->tcn_batches.push_back(batches[i]);
            }
        }
        if (!b->plans.empty()) {
            autotune(*b);
            layout(*b);
        }
        if (!b->nm_plans.empty()) layout_nm(*b);
        if (!b->jg_plans.empty()) b->jgroup = jit_group_create(b->jg_plans, b->jg_batches);
        if (!wide_plans.empty()) b->wide = wide_batch_create(wide_plans, wide_batches);
        if (!b->tc_plans.empty()) b->tcb = tc_batch_create(b->tc_plans, b->tc_batches, b->precision);
        if (!b->tcn_plans.empty()) b->tcnb = tcn_batch_create(b->tcn_plans, b->tcn_batches, b->precision);
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
            if ((b->kind[i] == 2 || b->kind[i] == 3) && x[i] == y[i])
                fail(GFT_ERR_UNSUPPORTED, "tensor-core entries do not run in place");
        }
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        const bool same = b->last_x.size() == (size_t)k &&
                          std::equal(x, x + k, b->last_x.begin()) &&
                          std::equal(y, y + k, b->last_y.begin(), [](float* a, const void* c) { return a == c; });
        if (!same) {
            // every group reads its signal pointers from device descriptors,
            // so the captured graph stays valid
            std::vector<const float*> tx, wx, cx, nx, mx, gx;
            std::vector<float*> ty, wy, cy, ny, my, gy;
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
            for (int i : b->tcn_users) {
                nx.push_back(x[i]);
                ny.push_back(y[i]);
            }
            for (int i : b->nm_users) {
                mx.push_back(x[i]);
                my.push_back(y[i]);
            }
            for (int i : b->jg_users) {
                gx.push_back(x[i]);
                gy.push_back(y[i]);
            }
            if (!b->plans.empty()) upload_desc(*b, tx.data(), ty.data(), st);
            if (!b->nm_plans.empty()) upload_classes(b->nm_classes, mx.data(), my.data(), st);
            if (b->jgroup) jit_group_upload(b->jgroup, gx, gy, st);
            if (b->wide) wide_batch_upload(b->wide, wx, wy, st);
            if (b->tcb) tc_batch_upload(b->tcb, cx, cy, st);
            if (b->tcnb) tcn_batch_upload(b->tcnb, nx, ny, st);
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
                bool used[gft_batch_s::kSide] = {};
                auto fork = [&](int s) {
                    if (!used[s]) GFT_CUDA(cudaStreamWaitEvent(b->side[s], b->ev_fork, 0));
                    used[s] = true;
                    return b->side[s];
                };
                if (b->wide) wide_batch_launch(b->wide, fork(0));
                // both tensor-core groups on one side stream: their CTAs
                // would otherwise compete for the SMs' TMEM
                if (b->tcb) tc_batch_launch(b->tcb, fork(1));
                if (b->tcnb) tcn_batch_launch(b->tcnb, fork(1));
                // the CUDA-core size classes one after another on the capture
                // stream (launched concurrently they take the SMs' shared
                // memory that the tensor-core kernels wait for)
                auto class_stream = [&](int) { return cs; };
                if (b->jgroup) jit_group_launch(b->jgroup, cs);
                if (!b->nm_plans.empty()) launch_nm(*b, class_stream);
                if (!b->plans.empty()) launch_batch(*b, class_stream);
                for (int s = 0; s < gft_batch_s::kSide; ++s)
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
        } else if (b->kind[i] == 4) {
            *tile = nm_ts(b->nm_plans[b->idx[i]]->n);
            *threads = kNmThreads;
        } else if (b->kind[i] == 5) {
            *tile = jit_group_tile(b->jgroup, b->idx[i]);
            *threads = 128;
        }
    });
}

gft_status gft_batch_get_launches(gft_batch_t b, int32_t* launches) {
    return guard_b([&] {
        if (!b || !launches) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        int32_t n = 0;
        for (auto& c : b->classes) n += c.total_items > 0 ? 1 : 0;
        for (auto& c : b->nm_classes) n += c.total_items > 0 ? 1 : 0;
        if (b->jgroup) n += jit_group_launches(b->jgroup);
        if (b->wide) n += wide_batch_launches(b->wide);
        if (b->tcb) n += tc_batch_launches(b->tcb);
        if (b->tcnb) n += tcn_batch_launches(b->tcnb);
        *launches = n;
    });
}

gft_status gft_batch_destroy(gft_batch_t b) {
    return guard_b([&] { delete b; });
}

}  // extern "C"

// CUDA-core transform kernel for plans with WIDE leaves (more than 32 nodes),
// FP32 and FP64, forward and inverse.
//
// The table-driven kernel (apply.cu) gives every thread whole signals: a
// thread gathers a leaf's m inputs into registers and computes all m
// outputs, so its registers and its shared-memory tile grow with m and the
// SM runs few warps once leaves reach 64 nodes.  Here the leaf products of
// a tile are instead computed like a small GEMM by the whole CTA:
//
//   Y_k[TS x m] = V_k[TS x m] * M_k[m x m]        (forward, Eq. 13 per leaf)
//
// with V_k the tile's post-stage values at the leaf's node slots.
//
// The tile is kept TRANSPOSED in shared memory, node-major: T[slot][signal]
// with a signal stride TSP (TS rounded up so rows are 16-byte aligned and
// sit 4 banks apart).  Then
//   * a Haar unit (x_i, x_j) -> (x_i + x_j, x_i - x_j) (Sec. III; the
//     1/sqrt2 factors are folded into M_k) is two 16-byte row loads and two
//     stores for four signals,
//   * the GEMM reads RS consecutive signals of one slot with vector loads
//     (a broadcast within a signal group) and OC entries of one matrix row
//     with vector loads (consecutive across the group's lanes), then issues
//     RS*OC FMAs -- about one shared-memory wavefront per 4-10 FMA
//     instructions, so the FMA pipe, not shared memory, is the limit,
//   * a leaf's outputs overwrite its own input slots (16-byte stores) once
//     every warp has finished reading them.
// Each thread owns an RS x OC register block; a warp is LR x LC threads
// (LC = P / OC output groups, P = leaf width rounded up to a power of two,
// LR = 32 / LC signal groups); the 4 warps cover TS = 4 * RS * LR signals.
// (RS, OC) is chosen per leaf on the host.  The leaf matrix streams from
// global memory (L2-resident) through two shared-memory chunk buffers with
// cp.async.  The tile itself arrives with 4-byte cp.async copies that
// transpose on the fly (a warp copies an 8-node x 4-signal block: one
// sector per signal row in global memory, 32 distinct banks in shared
// memory); the permuted store gathers four coefficients per thread and
// writes them with one 16-byte store.  The inverse loads through the
// permutation, runs the leaves with M_k^T and then the stages in reverse.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <vector>

#include "apply_core.cuh"

namespace gft {
using namespace core;
namespace {

constexpr int kWThreads = 128;
constexpr int kWSmemLimit = 232448;
constexpr int kWDesc = 8;   // per leaf: m, P, lab_off, f_off, i_off, variant, lc, kc_rows

struct WArgs {
    const void* x;
    void* y;
    const int* ints;       // plan program (pairs, stage offsets, labels, out_pos, src, ...)
    const int* wdesc;      // per-leaf descriptors, kWDesc ints each
    const void* mats;      // per leaf: M_f (m x P) then M_i (m x P), zero padded columns
    long long batch;
    int n, tsp, ts, nbuf, n_pairs, n_stages, n_leaves;
    int n_pre_stages;      // stages before the leaf products; the rest act on leaf outputs (right Haar units)
    int off_labels, off_src;
    int chunk_elems;       // elements of one matrix chunk buffer
    int inverse;
};

// W consecutive elements of shared memory into registers (vector loads)
template <class T, int W>
__device__ __forceinline__ void lds_vec(const T* p, T* w) {
    if constexpr (sizeof(T) == 4 && W % 4 == 0) {
#pragma unroll
        for (int q = 0; q < W / 4; ++q) {
            const float4 v = reinterpret_cast<const float4*>(p)[q];
            w[4 * q] = v.x;
            w[4 * q + 1] = v.y;
            w[4 * q + 2] = v.z;
            w[4 * q + 3] = v.w;
        }
    } else if constexpr (sizeof(T) == 4 && W == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        w[0] = v.x;
        w[1] = v.y;
    } else if constexpr (sizeof(T) == 8 && W % 2 == 0) {
#pragma unroll
        for (int q = 0; q < W / 2; ++q) {
            const double2 v = reinterpret_cast<const double2*>(p)[q];
            w[2 * q] = v.x;
            w[2 * q + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < W; ++q) w[q] = p[q];
    }
}

template <class T, int W>
__device__ __forceinline__ void sts_vec(T* p, const T* w) {
    if constexpr (sizeof(T) == 4 && W % 4 == 0) {
#pragma unroll
        for (int q = 0; q < W / 4; ++q)
            reinterpret_cast<float4*>(p)[q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    } else if constexpr (sizeof(T) == 4 && W == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(w[0], w[1]);
    } else if constexpr (sizeof(T) == 8 && W % 2 == 0) {
#pragma unroll
        for (int q = 0; q < W / 2; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(w[2 * q], w[2 * q + 1]);
    } else {
#pragma unroll
        for (int q = 0; q < W; ++q) p[q] = w[q];
    }
}

// rows x P elements of a leaf matrix (contiguous) -> shared memory, 16-byte
// copies (P * sizeof(T) is a multiple of 16 and chunks start 16-byte aligned)
template <class T>
__device__ __forceinline__ void load_chunk(T* dst, const T* src, int elems) {
    constexpr int PER = 16 / sizeof(T);
    for (int c = threadIdx.x; c < elems / PER; c += kWThreads) cp_async16(dst + c * PER, src + c * PER);
}

// One leaf's product over the tile, in place.  M points at the leaf's
// m x P matrix for this direction.  Thread (lr, lcol) of its warp owns the
// RS signals s0 .. s0+RS-1 and the OC output columns VW*(lcol + LC*q) + e
// (q < OC/VW, e < VW): every vector load of a matrix row is contiguous
// across the LC lanes of a signal group.  The next row's operands are
// loaded before the current row's FMAs are issued.
template <class T, int RS, int OC>
__device__ __forceinline__ void wide_leaf(T* tile, int tsp, int ts, const int* lab, const T* __restrict__ M, int m,
                                          int P, int lc, int kc_rows, T* mbuf, int chunk_elems) {
    constexpr int VE = 16 / sizeof(T);                   // elements per 16-byte vector
    constexpr int VW = OC < VE ? OC : VE;                 // matrix vector width
    constexpr int NV = OC / VW;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lr_cnt = 32 / lc;
    const int lr = lane / lc;
    const int lcol = lane - lr * lc;
    const int s0 = (warp * lr_cnt + lr) * RS;
    const bool live = s0 < ts;                            // tiles smaller than the CTA's cover
    const int sv = live ? s0 : 0;                          // reads stay inside the tile
    T acc[RS][OC];
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < OC; ++j) acc[i][j] = T(0);
    const int nch = (m + kc_rows - 1) / kc_rows;
    load_chunk(mbuf, M, min(kc_rows, m) * P);
    cp_async_commit();
    for (int kc = 0; kc < nch; ++kc) {
        if (kc + 1 < nch) {
            const int r0n = (kc + 1) * kc_rows;
            load_chunk(mbuf + ((kc + 1) & 1) * chunk_elems, M + (size_t)r0n * P, min(kc_rows, m - r0n) * P);
        }
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();   // chunk kc visible to every thread
        const T* Mc = mbuf + (kc & 1) * chunk_elems + VW * lcol;
        const int r0 = kc * kc_rows, rn = min(kc_rows, m - r0);
        const int* lab_c = lab + r0;
        // two register sets used in turn: the loads of row r+1 go to one set
        // while the FMAs of row r read the other (no register copies)
        T v0[RS], w0[OC], v1[RS], w1[OC];
        lds_vec<T, RS>(tile + lab_c[0] * tsp + sv, v0);
#pragma unroll
        for (int q = 0; q < NV; ++q) lds_vec<T, VW>(Mc + q * VW * lc, w0 + q * VW);
        int r = 0;
        for (; r + 1 < rn; r += 2) {
            lds_vec<T, RS>(tile + lab_c[r + 1] * tsp + sv, v1);
#pragma unroll
            for (int q = 0; q < NV; ++q) lds_vec<T, VW>(Mc + (r + 1) * P + q * VW * lc, w1 + q * VW);
#pragma unroll
            for (int i = 0; i < RS; ++i)
#pragma unroll
                for (int j = 0; j < OC; ++j) acc[i][j] = fma(v0[i], w0[j], acc[i][j]);
            const int r2 = min(r + 2, rn - 1);   // past the end: re-reads row rn-1 (in bounds, unused)
            lds_vec<T, RS>(tile + lab_c[r2] * tsp + sv, v0);
#pragma unroll
            for (int q = 0; q < NV; ++q) lds_vec<T, VW>(Mc + r2 * P + q * VW * lc, w0 + q * VW);
#pragma unroll
            for (int i = 0; i < RS; ++i)
#pragma unroll
                for (int j = 0; j < OC; ++j) acc[i][j] = fma(v1[i], w1[j], acc[i][j]);
        }
        if (r < rn) {   // odd row count: the last row is in set 0
#pragma unroll
            for (int i = 0; i < RS; ++i)
#pragma unroll
                for (int j = 0; j < OC; ++j) acc[i][j] = fma(v0[i], w0[j], acc[i][j]);
        }
        __syncthreads();   // every thread done with chunk kc's buffer and (last chunk) with V_k
    }
    if (live) {
#pragma unroll
        for (int q = 0; q < NV; ++q)
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const int c = VW * (lcol + lc * q) + e;
                if (c < m) {
                    T col[RS];
#pragma unroll
                    for (int i = 0; i < RS; ++i) col[i] = acc[i][q * VW + e];
                    sts_vec<T, RS>(tile + lab[c] * tsp + s0, col);
                }
            }
    }
}

// variant code = log2(RS) * 5 + log2(OC), RS in {1,2,4,8}, OC in {1,...,16}
template <class T>
__device__ __forceinline__ void wide_leaf_dispatch(int code, T* tile, int tsp, int ts, const int* lab, const T* M,
                                                   int m, int P, int lc, int kc, T* mbuf, int ce) {
#define GFT_W(R, O, C)                                                              \
    case C:                                                                        \
        if constexpr (sizeof(T) == 4 || R * O <= 32)                               \
            wide_leaf<T, R, O>(tile, tsp, ts, lab, M, m, P, lc, kc, mbuf, ce);     \
        break;
    switch (code) {
        GFT_W(1, 1, 0) GFT_W(1, 2, 1) GFT_W(1, 4, 2) GFT_W(1, 8, 3) GFT_W(1, 16, 4)
        GFT_W(2, 1, 5) GFT_W(2, 2, 6) GFT_W(2, 4, 7) GFT_W(2, 8, 8) GFT_W(2, 16, 9)
        GFT_W(4, 1, 10) GFT_W(4, 2, 11) GFT_W(4, 4, 12) GFT_W(4, 8, 13) GFT_W(4, 16, 14)
        GFT_W(8, 1, 15) GFT_W(8, 2, 16) GFT_W(8, 4, 17) GFT_W(8, 8, 18)
        default: break;
    }
#undef GFT_W
}

// One stage of Haar units on the transposed tile: thread -> (pair, 4 or 2
// consecutive signals), 16-byte row loads and stores.
template <class T>
__device__ __forceinline__ void wide_stage(T* tile, int tsp, int ts, const int* pairs, int p0, int P) {
    constexpr int VE = 16 / sizeof(T);
    const int groups = ts / VE;
    const int total = P * groups;
    for (int idx = threadIdx.x; idx < total; idx += kWThreads) {
        const int q = idx / groups;
        const int sg = idx - q * groups;
        const int i = pairs[2 * (p0 + q)], j = pairs[2 * (p0 + q) + 1];
        T u[VE], v[VE], a[VE], b[VE];
        lds_vec<T, VE>(tile + i * tsp + VE * sg, u);
        lds_vec<T, VE>(tile + j * tsp + VE * sg, v);
#pragma unroll
        for (int e = 0; e < VE; ++e) {
            a[e] = u[e] + v[e];
            b[e] = u[e] - v[e];
        }
        sts_vec<T, VE>(tile + i * tsp + VE * sg, a);
        sts_vec<T, VE>(tile + j * tsp + VE * sg, b);
    }
}

// Tile load, transposing: element (signal s, node j) -> T[slot(j)][s] with
// slot(j) = j (forward) or src[j] (inverse: coefficient j belongs to slot
// src[j]).  A warp moves an 8-node x 4-signal block per step.
template <class T>
__device__ __forceinline__ void wide_load(const WArgs& a, const int* src_slot, T* buf, long long tile) {
    const int rows = (int)min((long long)a.ts, a.batch - tile * (long long)a.ts);
    const T* src = reinterpret_cast<const T*>(a.x) + tile * (long long)a.ts * a.n;
    const int jb = (a.n + 7) >> 3, sb = (rows + 3) >> 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int jl = lane & 7, sl = lane >> 3;
    for (int blk = warp; blk < jb * sb; blk += kWThreads / 32) {
        const int bs = blk / jb;
        const int j = (blk - bs * jb) * 8 + jl, s = bs * 4 + sl;
        if (j < a.n && s < rows) cp_async_elem(buf + (a.inverse ? src_slot[j] : j) * a.tsp + s, src + (long long)s * a.n + j);
    }
}

// Tile store: forward y[s][j] = T[src[j]][s]; inverse x[s][j] = T[j][s].
// Four consecutive outputs per thread, one 16-byte (two for FP64) store.
template <class T>
__device__ __forceinline__ void wide_store(const WArgs& a, const int* src_slot, const T* buf, long long tile) {
    const long long rows = min((long long)a.ts, a.batch - tile * (long long)a.ts);
    T* dst = reinterpret_cast<T*>(a.y) + tile * (long long)a.ts * a.n;
    const int E = (int)rows * a.n;
    const bool fwd = !a.inverse;
    if (a.n % 4 == 0) {
        const int per_row = a.n / 4;
        for (int c = threadIdx.x; c < E / 4; c += kWThreads) {
            const int s = c / per_row;
            const int j = 4 * (c - s * per_row);
            T v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = buf[(fwd ? src_slot[j + q] : j + q) * a.tsp + s];
            Vec4Store<T>::st(dst + 4 * (long long)c, v[0], v[1], v[2], v[3]);
        }
    } else {
        for (int e = threadIdx.x; e < E; e += kWThreads) {
            const int s = e / a.n;
            const int j = e - s * a.n;
            __stcs(dst + e, buf[(fwd ? src_slot[j] : j) * a.tsp + s]);
        }
    }
}

// Tables of one plan in shared memory:
// [pairs 2P][stage_off S+1][labels n][src n][leaf desc kWDesc*L]
__device__ __forceinline__ void wide_load_tables(const WArgs& a, int* s_ints) {
    const int head = 2 * a.n_pairs + a.n_stages + 1;
    int* s_lab = s_ints + head;
    int* s_src = s_lab + a.n;
    int* s_desc = s_src + a.n;
    for (int i = threadIdx.x; i < head; i += kWThreads) s_ints[i] = a.ints[i];
    for (int i = threadIdx.x; i < a.n; i += kWThreads) {
        s_lab[i] = a.ints[a.off_labels + i];
        s_src[i] = a.ints[a.off_src + i];
    }
    for (int i = threadIdx.x; i < kWDesc * a.n_leaves; i += kWThreads) s_desc[i] = a.wdesc[i];
}

// Stages and leaf products of one tile already in shared memory.  Forward:
// left stages, leaves, right Haar units (bipartite plans); inverse: right
// units, leaves, left stages in reverse.  Ends with a barrier, so the tile
// is ready for the store.
template <class T>
__device__ __forceinline__ void wide_compute(const WArgs& a, T* buf, T* mbuf, const int* s_ints) {
    const int* s_pairs = s_ints;
    const int* s_soff = s_pairs + 2 * a.n_pairs;
    const int* s_lab = s_soff + a.n_stages + 1;
    const int* s_desc = s_lab + 2 * a.n;
    const T* mats = reinterpret_cast<const T*>(a.mats);
    const int pre = a.n_pre_stages;
    const int s0 = a.inverse ? a.n_stages - 1 : 0, s1 = a.inverse ? pre - 1 : pre, ds = a.inverse ? -1 : 1;
    for (int s = s0; s != s1; s += ds) {   // left stages (forward) / right units (inverse)
        wide_stage(buf, a.tsp, a.ts, s_pairs, s_soff[s], s_soff[s + 1] - s_soff[s]);
        __syncthreads();
    }
    for (int k = 0; k < a.n_leaves; ++k) {
        const int* d = s_desc + kWDesc * k;
        const T* M = mats + (a.inverse ? d[4] : d[3]);
        wide_leaf_dispatch<T>(d[5], buf, a.tsp, a.ts, s_lab + d[2], M, d[0], d[1], d[6], d[7], mbuf, a.chunk_elems);
    }
    __syncthreads();   // every leaf's outputs written
    const int t0 = a.inverse ? pre - 1 : pre, t1 = a.inverse ? -1 : a.n_stages;
    for (int s = t0; s != t1; s += ds) {   // right units (forward) / left stages in reverse (inverse)
        wide_stage(buf, a.tsp, a.ts, s_pairs, s_soff[s], s_soff[s + 1] - s_soff[s]);
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(kWThreads, 2) gft_wide_kernel(WArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [nbuf tiles][2 matrix chunks][tables]
    T* tiles = reinterpret_cast<T*>(smem_raw);
    const int tile_elems = a.n * a.tsp;
    T* mbuf = tiles + a.nbuf * tile_elems;
    int* s_ints = reinterpret_cast<int*>(mbuf + 2 * a.chunk_elems);
    const int* s_src = s_ints + 2 * a.n_pairs + a.n_stages + 1 + a.n;
    wide_load_tables(a, s_ints);
    __syncthreads();
    const long long n_tiles = (a.batch + a.ts - 1) / a.ts;
    long long tile = blockIdx.x;
    if (tile < n_tiles) wide_load<T>(a, s_src, tiles, tile);
    cp_async_commit();
    int cur = 0;
    for (; tile < n_tiles; tile += gridDim.x) {
        T* buf = tiles + cur * tile_elems;
        const long long nxt = tile + gridDim.x;
        if (a.nbuf == 2) {
            if (nxt < n_tiles) wide_load<T>(a, s_src, tiles + (cur ^ 1) * tile_elems, nxt);
            cp_async_commit();
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        __syncthreads();   // tile landed
        wide_compute<T>(a, buf, mbuf, s_ints);
        wide_store<T>(a, s_src, buf, tile);
        __syncthreads();   // buffer free
        if (a.nbuf == 2) {
            cur ^= 1;
        } else {
            if (nxt < n_tiles) wide_load<T>(a, s_src, tiles, nxt);
            cp_async_commit();
        }
    }
    cp_async_wait0();
}

// Mixed batches: one persistent launch over (plan, tile) items of many
// wide-leaf plans (FP32 forward).  Every CTA takes the next item from a
// device counter, finds its plan by binary search over the plans' first item
// indices, reloads the plan's tables into shared memory when the plan
// changes, and runs the single-plan tile code.
struct WBatchPlan {
    WArgs a;
    long long item0;
};

__global__ void __launch_bounds__(kWThreads, 2) gft_wide_batch_kernel(const WBatchPlan* __restrict__ plans, int n_plans,
                                                                   long long total_items,
                                                                   unsigned long long* counter, int tile_cap,
                                                                   int chunk_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* buf = reinterpret_cast<float*>(smem_raw);
    float* mbuf = buf + tile_cap;
    int* s_ints = reinterpret_cast<int*>(mbuf + 2 * chunk_cap);
    __shared__ long long s_item;
    __shared__ int s_plan;
    int loaded = -1;
    while (true) {
        if (threadIdx.x == 0) {
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
        const WArgs a = plans[p].a;
        if (p != loaded) {
            wide_load_tables(a, s_ints);
            __syncthreads();
            loaded = p;
        }
        const int* s_src = s_ints + 2 * a.n_pairs + a.n_stages + 1 + a.n;
        const long long tile = it - plans[p].item0;
        wide_load<float>(a, s_src, buf, tile);
        cp_async_commit();
        cp_async_wait0();
        __syncthreads();
        wide_compute<float>(a, buf, mbuf, s_ints);
        wide_store<float>(a, s_src, buf, tile);
        __syncthreads();   // tile buffer and s_item free
    }
}

int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}
int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// Signal stride of the transposed tile: a multiple of the 16-byte vector
// (rows stay aligned) that is 4 (mod 8) floats, so the 8-node x 4-signal
// blocks of the tile load hit 32 distinct banks; FP64: 2 (mod 4).
int signal_stride(int ts, size_t esz) {
    if (esz == 4) return ts % 8 == 0 ? ts + 4 : ts + 8;
    return ts % 4 == 0 ? ts + 2 : ts + 4;
}

struct WVariant {
    int rs, oc, lc;
};

// (RS, OC) for a leaf of padded width P in a tile of TS signals; rs = 0 if none
WVariant pick_variant(int P, int ts, size_t esz) {
    const int max_acc = esz == 4 ? 64 : 32;
    const int target = ts * P / 128;
    if (target < 1) return P <= 32 ? WVariant{1, 1, P} : WVariant{0, 0, 0};
    if (target > max_acc) return {0, 0, 0};
    const int vw = 16 / (int)esz;
    WVariant best{0, 0, 0};
    double best_ratio = -1.0;
    for (int rs = 1; rs <= 8; rs <<= 1) {
        if (target % rs) continue;
        const int oc = target / rs;
        if (oc > 16 || oc > P || (rs == 8 && oc == 16)) continue;
        const int lc = P / oc;
        if (lc < 1 || lc > 32) continue;
        const int vloads = std::max(1, oc / vw);
        const double m_wave = vloads * std::max(1.0, lc * (double)std::min(oc, vw) * esz / 128.0);
        const double v_wave = std::max(1, rs / vw);   // broadcast within a signal group
        const double ratio = (double)(rs * oc) / (v_wave + m_wave);
        if (ratio > best_ratio) {
            best_ratio = ratio;
            best = {rs, oc, lc};
        }
    }
    return best;
}

struct WidePlan {
    struct Cfg {
        int ts = 0, nbuf = 1, chunk_elems = 0;
        size_t smem = 0;
        int* d_desc = nullptr;
        bool use = false;          // chosen over the table-driven kernel
    } cfg[2];                      // FP32, FP64
    float* d_m32 = nullptr;
    double* d_m64 = nullptr;
    ~WidePlan() {
        for (auto& c : cfg)
            if (c.d_desc) cudaFree(c.d_desc);
        if (d_m32) cudaFree(d_m32);
        if (d_m64) cudaFree(d_m64);
    }
};

}  // namespace

template <class T>
static void launch_wide_t(gft_plan_s& p, const T* x, T* y, int64_t batch, bool inverse, cudaStream_t st);
static void wide_tune(gft_plan_s& p);

bool wide_eligible(const gft_plan_s& p) {
    int mx = 0;
    for (auto& lf : p.leaves) mx = std::max(mx, lf.m());
    return p.n >= 4 && mx > 32 && mx <= 512;
}

// Host preparation: pow2-padded forward / inverse leaf matrices (FP32 and
// FP64) and, per precision, the tile size and per-leaf variants.
void wide_build(gft_plan_s& p) {
    if (!wide_eligible(p)) return;
    WidePlan* W = new WidePlan;
    try {
        const int n = p.n;
        std::vector<double> mats;
        std::vector<int> Ps, lab_off, f_off, i_off;
        int lo = 0;
        for (auto& lf : p.leaves) {
            const int m = lf.m(), P = std::max(4, pow2_at_least(m));
            Ps.push_back(P);
            lab_off.push_back(lo);
            lo += m;
            f_off.push_back((int)mats.size());
            std::vector<double> Mf((size_t)m * P, 0.0), Mi((size_t)m * P, 0.0);
            for (int r = 0; r < m; ++r) {
                for (int c = 0; c < m; ++c) {
                    const double v = lf.fold(r, c);
                    Mf[(size_t)r * P + c] = v;   // forward: y_c = sum_r v_r Mf[r][c]
                    Mi[(size_t)c * P + r] = v;   // inverse: x_r = sum_c y_c Mi[c][r]
                }
            }
            mats.insert(mats.end(), Mf.begin(), Mf.end());
            i_off.push_back((int)mats.size());
            mats.insert(mats.end(), Mi.begin(), Mi.end());
        }
        const int ints_smem = 2 * p.dev.n_pairs + p.dev.n_stages + 1 + 2 * n + kWDesc * (int)p.leaves.size();
        for (int prec = 0; prec < 2; ++prec) {
            const size_t esz = prec == 0 ? 4 : 8;
            int maxP = 4;
            for (int P : Ps) maxP = std::max(maxP, P);
            WidePlan::Cfg& c = W->cfg[prec];
            // largest power-of-two tile (64 down to 4) whose leaves all have a
            // variant and whose buffers fit; two tile buffers when they fit
            // in about half of the SM (two CTAs per SM) or when the tile is small
            for (int ts = 64; ts >= 4; ts >>= 1) {
                bool ok = true;
                int chunk = 0;
                std::vector<int> desc;
                for (size_t k = 0; k < p.leaves.size() && ok; ++k) {
                    const int m = p.leaves[k].m(), P = Ps[k];
                    const WVariant v = pick_variant(P, ts, esz);
                    if (!v.rs) {
                        ok = false;
                        break;
                    }
                    int kc = std::max(4, (int)(16384 / (P * esz)));
                    kc = std::min(kc, m);
                    chunk = std::max(chunk, kc * P);
                    desc.insert(desc.end(), {m, P, lab_off[k], f_off[k], i_off[k],
                                             ilog2(v.rs) * 5 + ilog2(v.oc), v.lc, kc});
                }
                if (!ok) continue;
                const size_t fixed = esz * 2 * (size_t)chunk + sizeof(int) * (size_t)((ints_smem + 3) & ~3);
                const size_t tile = esz * (size_t)n * signal_stride(ts, esz);
                int nbuf = 0;
                if (fixed + 2 * tile <= (size_t)kWSmemLimit / 2 - 1024) nbuf = 2;
                else if (fixed + tile <= (size_t)kWSmemLimit) nbuf = 1;
                if (!nbuf) continue;
                if (const char* e = std::getenv("GFT_WIDE_TS")) {
                    const int want = std::atoi(e);
                    if (want && want != ts) continue;
                }
                c.ts = ts;
                c.nbuf = nbuf;
                c.chunk_elems = chunk;
                c.smem = fixed + nbuf * tile;
                GFT_CUDA(cudaMalloc(&c.d_desc, sizeof(int) * desc.size()));
                GFT_CUDA(cudaMemcpy(c.d_desc, desc.data(), sizeof(int) * desc.size(), cudaMemcpyHostToDevice));
                break;
            }
        }
        std::vector<float> m32(mats.begin(), mats.end());
        GFT_CUDA(cudaMalloc(&W->d_m32, sizeof(float) * m32.size()));
        GFT_CUDA(cudaMemcpy(W->d_m32, m32.data(), sizeof(float) * m32.size(), cudaMemcpyHostToDevice));
        GFT_CUDA(cudaMalloc(&W->d_m64, sizeof(double) * mats.size()));
        GFT_CUDA(cudaMemcpy(W->d_m64, mats.data(), sizeof(double) * mats.size(), cudaMemcpyHostToDevice));
    } catch (...) {
        delete W;
        throw;
    }
    p.wide = W;
    // Choose between this kernel and the table-driven one (which handles
    // leaves up to 64 nodes) by timing both on a scratch batch.
    // GFT_KERNEL_TABLE keeps the table-driven kernel wherever it fits.
    bool tune = false;
    for (int prec = 0; prec < 2; ++prec) {
        WidePlan::Cfg& c = W->cfg[prec];
        const bool table_ok = apply_supported(apply_args(p, prec == 1), prec == 1);
        c.use = c.ts > 0 && (!table_ok || !(p.flags & GFT_KERNEL_TABLE));
        tune |= c.use && table_ok && !(p.flags & GFT_KERNEL_WIDE);
    }
    if (tune) wide_tune(p);
}

void wide_free(gft_plan_s& p) {
    delete static_cast<WidePlan*>(p.wide);
    p.wide = nullptr;
}

bool wide_configured(const gft_plan_s& p) {
    const WidePlan* W = static_cast<const WidePlan*>(p.wide);
    return W && W->cfg[0].ts > 0;
}

bool wide_ready(const gft_plan_s& p, bool f64) {
    const WidePlan* W = static_cast<const WidePlan*>(p.wide);
    return W && W->cfg[f64 ? 1 : 0].use;
}

// Time the wide and the table-driven FP32 / FP64 forward kernels on a
// scratch batch of zeros (no data-dependent work) and keep the faster.
static void wide_tune(gft_plan_s& p) {
    WidePlan* W = static_cast<WidePlan*>(p.wide);
    const int n = p.n;
    const int64_t tb = std::max<int64_t>(4096, (int64_t)(32 << 20) / (8 * n));
    void* dx = nullptr;
    void* dy = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    auto cleanup = [&] {
        if (dx) cudaFree(dx);
        if (dy) cudaFree(dy);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    };
    try {
        GFT_CUDA(cudaMalloc(&dx, (size_t)tb * n * 8));
        GFT_CUDA(cudaMalloc(&dy, (size_t)tb * n * 8));
        GFT_CUDA(cudaMemset(dx, 0, (size_t)tb * n * 8));
        GFT_CUDA(cudaEventCreate(&e0));
        GFT_CUDA(cudaEventCreate(&e1));
        GFT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        for (int prec = 0; prec < 2; ++prec) {
            if (!W->cfg[prec].use || !apply_supported(apply_args(p, prec == 1), prec == 1)) continue;
            float best[2] = {1e30f, 1e30f};
            for (int rep = 0; rep < 3; ++rep)
                for (int which = 0; which < 2; ++which) {
                    GFT_CUDA(cudaEventRecord(e0, st));
                    if (prec == 0) {
                        if (which) launch_wide_t<float>(p, (const float*)dx, (float*)dy, tb, false, st);
                        else launch_apply_f32(apply_args(p, false), (const float*)dx, (float*)dy, tb, false, st);
                    } else {
                        if (which) launch_wide_t<double>(p, (const double*)dx, (double*)dy, tb, false, st);
                        else launch_apply_f64(apply_args(p, true), (const double*)dx, (double*)dy, tb, false, st);
                    }
                    GFT_CUDA(cudaEventRecord(e1, st));
                    GFT_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    GFT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    best[which] = std::min(best[which], ms);
                }
            W->cfg[prec].use = best[1] < best[0];
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

template <class T>
static void launch_wide_t(gft_plan_s& p, const T* x, T* y, int64_t batch, bool inverse, cudaStream_t st) {
    WidePlan* W = static_cast<WidePlan*>(p.wide);
    const int prec = sizeof(T) == 8 ? 1 : 0;
    const auto& c = W->cfg[prec];
    if (!c.ts) fail(GFT_ERR_UNSUPPORTED, "no wide-leaf kernel configuration fits this plan");
    WArgs a{};
    a.x = x;
    a.y = y;
    a.ints = p.dev.d_ints;
    a.wdesc = c.d_desc;
    a.mats = prec ? (const void*)W->d_m64 : (const void*)W->d_m32;
    a.batch = batch;
    a.n = p.n;
    a.tsp = signal_stride(c.ts, sizeof(T));
    a.ts = c.ts;
    a.nbuf = c.nbuf;
    a.n_pairs = p.dev.n_pairs;
    a.n_stages = p.dev.n_stages;
    a.n_pre_stages = p.dev.n_pre_stages;
    a.n_leaves = p.dev.n_leaves;
    a.off_labels = 2 * p.dev.n_pairs + p.dev.n_stages + 1;
    a.off_src = a.off_labels + 2 * p.n;
    a.chunk_elems = c.chunk_elems;
    a.inverse = inverse ? 1 : 0;
    auto fn = gft_wide_kernel<T>;
    GFT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem));
    int per_sm = 0;
    GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kWThreads, c.smem));
    if (per_sm < 1) fail(GFT_ERR_UNSUPPORTED, "wide-leaf kernel does not fit on an SM");
    const long long n_tiles = (batch + c.ts - 1) / c.ts;
    const long long grid = std::min<long long>(n_tiles, (long long)per_sm * sm_count());
    fn<<<(unsigned)grid, kWThreads, c.smem, st>>>(a);
    GFT_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// mixed batches of wide-leaf plans (FP32 forward)
// ---------------------------------------------------------------------------
namespace {
struct WideBatch {
    std::vector<WBatchPlan> desc;   // slot order (decreasing cost per item)
    std::vector<int> order;         // slot -> index in the caller's list
    WBatchPlan* d_desc = nullptr;
    unsigned long long* d_counter = nullptr;
    long long total_items = 0;
    int tile_cap = 0, chunk_cap = 0;
    size_t smem = 0;
    int grid = 0;
    ~WideBatch() {
        if (d_desc) cudaFree(d_desc);
        if (d_counter) cudaFree(d_counter);
    }
};
}  // namespace

void* wide_batch_create(const std::vector<gft_plan_s*>& plans, const std::vector<int64_t>& batches) {
    std::unique_ptr<WideBatch> B(new WideBatch);
    const int k = (int)plans.size();
    std::vector<WBatchPlan> d(k);
    std::vector<double> cost(k);
    int ints_cap = 0;
    for (int i = 0; i < k; ++i) {
        gft_plan_s& p = *plans[i];
        WidePlan* W = static_cast<WidePlan*>(p.wide);
        if (!W || !W->cfg[0].ts) fail(GFT_ERR_UNSUPPORTED, "plan has no wide-leaf kernel configuration");
        const auto& c = W->cfg[0];
        WArgs& a = d[i].a;
        a = WArgs{};
        a.ints = p.dev.d_ints;
        a.wdesc = c.d_desc;
        a.mats = W->d_m32;
        a.batch = batches[i];
        a.n = p.n;
        a.tsp = signal_stride(c.ts, 4);
        a.ts = c.ts;
        a.nbuf = 1;
        a.n_pairs = p.dev.n_pairs;
        a.n_stages = p.dev.n_stages;
        a.n_pre_stages = p.dev.n_pre_stages;
        a.n_leaves = p.dev.n_leaves;
        a.off_labels = 2 * p.dev.n_pairs + p.dev.n_stages + 1;
        a.off_src = a.off_labels + 2 * p.n;
        a.chunk_elems = c.chunk_elems;
        a.inverse = 0;
        double fl = 0;
        for (auto& lf : p.leaves) fl += (double)lf.m() * lf.m();
        cost[i] = (fl + 8.0 * p.n) * c.ts;
        B->tile_cap = std::max(B->tile_cap, p.n * a.tsp);
        B->chunk_cap = std::max(B->chunk_cap, c.chunk_elems);
        ints_cap = std::max(ints_cap, 2 * a.n_pairs + a.n_stages + 1 + 2 * a.n + kWDesc * a.n_leaves);
    }
    B->order.resize(k);
    for (int i = 0; i < k; ++i) B->order[i] = i;
    std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int slot = 0; slot < k; ++slot) {
        WBatchPlan e = d[B->order[slot]];
        e.item0 = B->total_items;
        B->total_items += (e.a.batch + e.a.ts - 1) / e.a.ts;
        B->desc.push_back(e);
    }
    B->smem = sizeof(float) * ((size_t)B->tile_cap + 2 * (size_t)B->chunk_cap) + sizeof(int) * (size_t)ints_cap;
    if (B->smem > (size_t)kWSmemLimit) fail(GFT_ERR_UNSUPPORTED, "mixed batch of wide plans needs too much shared memory");
    GFT_CUDA(cudaMalloc(&B->d_desc, sizeof(WBatchPlan) * std::max(1, k)));
    GFT_CUDA(cudaMalloc(&B->d_counter, sizeof(unsigned long long)));
    GFT_CUDA(cudaFuncSetAttribute(gft_wide_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem));
    int per_sm = 0;
    GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gft_wide_batch_kernel, kWThreads, B->smem));
    if (per_sm < 1) fail(GFT_ERR_UNSUPPORTED, "wide mixed-batch kernel does not fit on an SM");
    B->grid = per_sm * sm_count();
    return B.release();
}

void wide_batch_upload(void* h, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st) {
    WideBatch* B = static_cast<WideBatch*>(h);
    for (size_t slot = 0; slot < B->desc.size(); ++slot) {
        B->desc[slot].a.x = x[B->order[slot]];
        B->desc[slot].a.y = y[B->order[slot]];
    }
    GFT_CUDA(cudaMemcpyAsync(B->d_desc, B->desc.data(), sizeof(WBatchPlan) * B->desc.size(), cudaMemcpyHostToDevice, st));
}

void wide_batch_launch(void* h, cudaStream_t st) {
    WideBatch* B = static_cast<WideBatch*>(h);
    GFT_CUDA(cudaMemsetAsync(B->d_counter, 0, sizeof(unsigned long long), st));
    if (B->total_items == 0) return;
    gft_wide_batch_kernel<<<B->grid, kWThreads, B->smem, st>>>(B->d_desc, (int)B->desc.size(), B->total_items,
                                                             B->d_counter, B->tile_cap, B->chunk_cap);
    GFT_CUDA(cudaGetLastError());
}

void wide_batch_free(void* h) { delete static_cast<WideBatch*>(h); }

int wide_batch_launches(void* h) { return static_cast<WideBatch*>(h)->total_items > 0 ? 1 : 0; }

void launch_wide_f32(gft_plan_s& p, const float* x, float* y, int64_t batch, bool inverse, cudaStream_t st) {
    launch_wide_t<float>(p, x, y, batch, inverse, st);
}
void launch_wide_f64(gft_plan_s& p, const double* x, double* y, int64_t batch, bool inverse, cudaStream_t st) {
    launch_wide_t<double>(p, x, y, batch, inverse, st);
}

}  // namespace gft

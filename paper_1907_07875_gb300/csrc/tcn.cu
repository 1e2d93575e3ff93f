// Tensor-core leaf products for batches of many graphs with FEW signals
// each (the size sweep: 10^4 graphs of 8..1024 nodes, a few dozen to a few
// hundred signals per graph), leaves up to 512 nodes.
//
// The leaf products y_k = M_k^T v_k (Sec. IV-C, Eq. 13; M_k the folded leaf
// basis) run with the roles of the operands swapped against tc.cu: the MMA's
// M axis is the leaf's output coefficients (128 per M-tile), its N axis the
// signals of a tile (NS = 16..128, the graph's whole batch when it fits), K
// the leaf's inputs:
//     D[c][s] (TMEM lane c, column s) = sum_r M_k[r][c] v_k[r][s]
// so a graph with 27 signals fills a 32-column accumulator instead of 27 of
// 128 rows, a 512-node leaf is four M-tiles, and each graph's basis crosses
// HBM once per tile of up to 128 signals.
//
// Two kernels per launch:
//   tcn_pack_kernel  (CTA per 8 signals of a tile): copies the rows into
//     shared memory (cp.async), computes the FP16 per-signal scales, runs
//     the Haar stages in place (FP32), and writes the B operand of every
//     (leaf, 32-wide K chunk) -- the gathered post-stage values split into
//     hi and lo (BF16 or scaled FP16) in the canonical no-swizzle K-major
//     core-matrix layout, NS rows per chunk -- to a scratch buffer, 512
//     contiguous bytes per 32 consecutive threads;
//   tcn_kernel  (persistent; work items = (plan, tile, group of M-tile
//     units), so a large graph's M-tiles spread over several SMs):
//     warp 8 (one thread) streams each step's basis chunk A = M_k^T (128
//     rows x 32 K, hi and lo) and signal chunk B (NS rows x 32 K, hi and lo)
//     through a ring of shared-memory slots with bulk copies (TMA);
//     warp 9 allocates TMEM (512 columns, two halves used by alternate
//     items) and one thread issues the MMAs (M = 128, N = NS, K = 16;
//     hi*hi + hi*lo + lo*hi for the split precisions) into one NS-column
//     accumulator per unit; warps 0-7 read a finished half (tcgen05.ld; the
//     two warps of a TMEM lane quarter split its columns), undo the FP16 scale and store each
//     coefficient at its output position (ascending eigenvalue) of its
//     signal's row, while the MMAs of the next item fill the other half;
//     the positions (a table of 128 per unit) and the scales of the next
//     item are staged into shared memory (cp.async) while this one is
//     stored.  A work item holds at most kNItemSteps / (K chunks of the
//     plan's widest leaf) units, so that a large graph spreads over many SMs.
// Every wait is bounded (about 2 s via %globaltimer); a timeout records
// GFT_ERR_TIMEOUT in the plan's error word, every role leaves its loop,
// copies and MMAs in flight are awaited (bounded), and TMEM is freed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "gft_internal.h"

namespace gft {
namespace {

constexpr int kNM = 128;             // coefficient rows per MMA (M)
constexpr int kNK = 32;              // K per chunk
constexpr int kNMaxNs = 128;         // signals per tile (MMA N)
constexpr int kNWorkers = 8;         // epilogue warps 0-7 (two per TMEM lane quarter)
constexpr int kNThreads = 320;       // + copier warp 8, MMA warp 9
constexpr int kNSlots = 4;           // ring slots (146 KB of shared memory with the static part: a CUDA-core CTA fits beside)
constexpr int kNCols = 512;          // TMEM columns per CTA (one CTA per SM): two halves
constexpr int kNHalf = 256;
constexpr int kNMaxLeaf = 512;
constexpr int kNItemSteps = 16;      // K chunks of the widest leaf per work item (at most)
constexpr unsigned kNAHalf = kNM * kNK * 2u;          // 8 KB: one of A hi / A lo
constexpr unsigned kNBHalf = kNMaxNs * kNK * 2u;      // 8 KB: one of B hi / B lo (at most)
constexpr unsigned kNSlotBytes = 2u * kNAHalf + 2u * kNBHalf;   // 32 KB
constexpr unsigned long long kNWaitNs = 2000000000ull;
constexpr int kPackThreads = 256;   // pack CTA: one group of 8 signals at a time
constexpr int kPackShortNp = 264;    // pack launch of short rows (n <= 260): many CTAs per SM

struct TcnLeaf {
    int m;          // leaf size
    int npad;       // rows of the basis image (m rounded up to 16)
    int kchunks;    // ceil(m / 32)
    int mtiles;     // ceil(npad / 128)
    int lab;        // offset of the leaf's nodes in the plan's leaf-ordered label / output-position lists
    int kc0;        // first chunk of this leaf in a tile's B image
    int unit0;      // first unit (M-tile) of this leaf
    int pad;
    long long a_off;   // element offset of the leaf's basis images
};

// one M-tile of a leaf (a unit): what the copier and the MMA issuer need
struct TcnUnit {
    long long a_off;   // element offset of this M-tile's rows in the leaf's first K chunk image
    int a_kstride;     // elements between consecutive K chunk images of the leaf (npad * 32)
    int abytes;        // bytes of one of A hi / A lo per chunk (rows * 32 * 2)
    int kchunks;       // K chunks of the leaf
    int kc0;           // the leaf's first chunk in a tile's B image
    int kmax;          // the leaf's K rounded up to 16
    int pad;
};

// one plan of a launch (an entry of the caller's batch)
struct TcnPlanDev {
    const float* x;
    float* y;
    long long batch;
    long long tile0;           // first tile of this plan in the launch
    long long item0;           // first work item of this plan in the launch
    const int* prog;           // [pairs 2P][stage offsets S+1][labels n][out_pos n] ...
    const TcnUnit* units;      // per unit (M-tile of a leaf)
    const int* upos;           // per unit 128 output positions (-1 past the leaf's end)
    const short* gather;       // per chunk 32 node labels (-1: padding), chunks in leaf order
    const unsigned char* ahi;  // basis images of this launch's precision
    const unsigned char* alo;
    unsigned char* bimg;       // B images of this plan's tiles (scratch): [tile][chunk][hi ns*64 B | lo]
    float* scale;              // per signal (scratch)
    int* err;                  // the plan's device error word
    int n, np, ns, n_units, n_chunks, n_stages, n_pairs;
    long long grp0;            // first 8-signal group of this plan in the launch (pack kernel)
    int upi;                   // units per work item
    int items_per_tile;
};

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// no-swizzle K-major descriptor: start, leading (K-group) byte offset,
// stride (8-row group) byte offset, version 1
__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulate, A/B BF16 or FP16,
// both K-major, N >> 3, M >> 4
__device__ __forceinline__ unsigned idesc(int n, bool bf16) {
    unsigned d = 1u << 4;
    if (bf16) d |= (1u << 7) | (1u << 10);
    d |= (unsigned)((n >> 3) & 0x3F) << 17;
    d |= (unsigned)((kNM >> 4) & 0x1F) << 24;
    return d;
}

__device__ __forceinline__ void mma(unsigned dt, unsigned long long ad, unsigned long long bd, unsigned id,
                                    unsigned acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void bar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok)
                 : "r"(su32(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool bar_wait(unsigned long long* b, unsigned parity) {
    if (bar_try(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    while (!bar_try(b, parity))
        if (now_ns() - t0 > kNWaitNs) return false;
    return true;
}
__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(b))
                 : "memory");
}
__device__ __forceinline__ void commit_to(unsigned long long* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}
// barrier 1 over the eight epilogue warps with an OR reduction: every one
// gets the same answer, so exits taken on it are uniform
__device__ __forceinline__ bool workers_any(bool v) {
    unsigned r;
    asm volatile("{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.or.pred q, 1, 256, p; selp.u32 %0, 1, 0, q; }"
                 : "=r"(r)
                 : "r"((unsigned)v)
                 : "memory");
    return r != 0;
}

// byte offset of (row, K group) in a [rows x 32] K-major no-swizzle image
// whose 8-row groups are 512 B apart (4 K groups of 16 B per row)
__device__ __forceinline__ unsigned coff(int row, int kg) {
    return (unsigned)(((row >> 3) * 4 + kg) * 128 + (row & 7) * 16);
}

// plan slot of work index v, walking forward from slot s (first indices in
// slot order): WHAT = 0 work items, 1 pack groups
template <int WHAT>
__device__ __forceinline__ int slot_of(const TcnPlanDev* P, int n_plans, int s, long long v) {
    while (s + 1 < n_plans && (WHAT == 0 ? P[s + 1].item0 : P[s + 1].grp0) <= v) ++s;
    return s;
}

}  // namespace
}  // namespace gft

namespace gft {
namespace {

// B images: one CTA (kPackThreads) per group of 8 signals (rows
// row0..row0+7 of tile t of a plan; rows past the batch are zeros); CTA b
// runs groups [range[b], range[b+1]) (first_slot[b]: the plan of the first).
// Warp r copies row r (cp.async, row stride np), takes its FP16 scale and
// runs the Haar stages on it (lanes over the units of a stage); after a
// barrier, thread (chunk, K group, row) gathers 8 post-stage values through
// the chunk's gather table and writes 16 B of hi and of lo of the B operand
// of every (leaf, K chunk), 32 consecutive threads covering 512 contiguous
// bytes.
__global__ void __launch_bounds__(kPackThreads) tcn_pack_kernel(const TcnPlanDev* __restrict__ plans, int n_plans,
                                                                const long long* __restrict__ range,
                                                                const int* __restrict__ first_slot, int prec) {
    extern __shared__ __align__(16) float buf[];
    __shared__ float s_inv[8];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool fp16 = prec == GFT_PREC_FP16X3, split = prec != GFT_PREC_BF16;
    int sl = first_slot[blockIdx.x];
    for (long long g = range[blockIdx.x]; g < range[blockIdx.x + 1]; ++g) {
        sl = slot_of<1>(plans, n_plans, sl, g);
        const TcnPlanDev& D = plans[sl];
        const int n = D.n, np = D.np, ns = D.ns, gpt = ns >> 3;
        const long long local = g - D.grp0;
        const long long t = local / gpt;
        const int rg = (int)(local - t * gpt);
        const long long row0 = t * ns + rg * 8;
        const int valid = (int)max(0LL, min(8LL, D.batch - row0));
        // warp r owns row r: its copy, its scale and its Haar stages need
        // only warp-level ordering
        float* row = buf + warp * np;
        if (warp < valid) {
            const float* src = D.x + (row0 + warp) * n;
            if ((n & 3) == 0) {
                for (int c4 = lane; 4 * c4 < n; c4 += 32)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(row + 4 * c4)),
                                 "l"(src + 4 * c4)
                                 : "memory");
            } else {
                for (int c = lane; c < n; c += 32)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(su32(row + c)), "l"(src + c)
                                 : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        // FP16: a power-of-two scale per signal bounding its post-stage values
        {
            float mx = 0.f;
            if (fp16 && warp < valid)
                for (int c = lane; c < n; c += 32) mx = fmaxf(mx, fabsf(row[c]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const float sc = mx > 0.f ? exp2f(ceilf(log2f(mx)) + (float)D.n_stages) : 1.f;
            if (lane == 0) {
                s_inv[warp] = 1.f / sc;
                if (warp < valid) D.scale[row0 + warp] = sc;
            }
        }
        // Haar stages in place (Sec. III; the 1/sqrt2 factors are in the
        // basis): the units of a stage touch disjoint nodes
        if (warp < valid) {
            const int* st_off = D.prog + 2 * D.n_pairs;
            for (int st = 0; st < D.n_stages; ++st) {
                const int p1 = st_off[st + 1];
                for (int pp = st_off[st] + lane; pp < p1; pp += 32) {
                    const int2 ij = *reinterpret_cast<const int2*>(D.prog + 2 * pp);
                    const float u = row[ij.x], v = row[ij.y];
                    row[ij.x] = u + v;
                    row[ij.y] = u - v;
                }
                __syncwarp();
            }
        }
        __syncthreads();   // scales and stages visible
        unsigned char* tb = D.bimg + (size_t)t * D.n_chunks * ns * 128;
        for (int e = tid; e < D.n_chunks * 32; e += kPackThreads) {
            const int r = e & 7, kg = (e >> 3) & 3, c = e >> 5;
            const bool live = r < valid;
            const float iv = s_inv[r];
            const float* rr = buf + r * np;
            const int4 g4 = *reinterpret_cast<const int4*>(D.gather + c * kNK + kg * 8);
            const short* gs = reinterpret_cast<const short*>(&g4);
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = (live && gs[q] >= 0) ? rr[gs[q]] * iv : 0.f;
            unsigned hi[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (fp16) {
                    const __half2 h = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
                    const float2 hf = __half22float2(h);
                    const __half2 l = __floats2half2_rn(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
                    hi[q] = *reinterpret_cast<const unsigned*>(&h);
                    lo[q] = *reinterpret_cast<const unsigned*>(&l);
                } else {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                    const float2 hf = __bfloat1622float2(h);
                    const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
                    hi[q] = *reinterpret_cast<const unsigned*>(&h);
                    lo[q] = *reinterpret_cast<const unsigned*>(&l);
                }
            }
            unsigned char* dst = tb + (size_t)c * ns * 128 + coff(rg * 8 + r, kg);
            __stcg(reinterpret_cast<uint4*>(dst), make_uint4(hi[0], hi[1], hi[2], hi[3]));
            if (split) __stcg(reinterpret_cast<uint4*>(dst + ns * 64), make_uint4(lo[0], lo[1], lo[2], lo[3]));
        }
        __syncthreads();   // buffer reusable
    }
}

// Work item i of a plan: tile t = i / items_per_tile, units
// [g * upi, min((g + 1) * upi, n_units)) with g = i % items_per_tile.
// CTA b runs items [range[b], range[b+1]) (first_slot[b]: plan of the first).
// Shared memory: kNSlots ring slots of [A hi | A lo | B hi | B lo], 8 KB each.
__global__ void __launch_bounds__(kNThreads, 1) tcn_kernel(const TcnPlanDev* __restrict__ plans, int n_plans,
                                                          const long long* __restrict__ range,
                                                          const int* __restrict__ first_slot, int prec) {
    extern __shared__ __align__(128) unsigned char ring[];
    __shared__ __align__(8) unsigned long long full[kNSlots], empty[kNSlots], acc_full[2], acc_free[2], drain;
    __shared__ float s_sc[2][kNMaxNs];   // per-signal scales of the items in the two TMEM halves
    __shared__ __align__(16) int s_pos[2][kNHalf / 16 * kNM];   // their output positions (at most 16 units)
    __shared__ unsigned s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == kNWorkers + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"(kNCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kNSlots; ++i) {
            bar_init(&full[i], 1);
            bar_init(&empty[i], 1);
        }
        for (int h = 0; h < 2; ++h) {
            bar_init(&acc_full[h], 1);
            bar_init(&acc_free[h], kNWorkers);
        }
        bar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    const bool split = prec != GFT_PREC_BF16;
    const bool fp16 = prec == GFT_PREC_FP16X3;
    const long long i0 = range[blockIdx.x], i1 = range[blockIdx.x + 1];
    const int slot0 = first_slot[blockIdx.x];
    auto abort_now = [&](int* err) {
        s_abort = 1;
        atomicExch(err, (int)GFT_ERR_TIMEOUT);
    };

    if (warp == kNWorkers) {
        // ---------------- copies (TMA) ----------------
        if (lane == 0) {
            long long q = 0;
            bool issued[kNSlots] = {};
            unsigned par[kNSlots] = {};
            bool stop = false;
            int sl = slot0;
            for (long long it = i0; it < i1 && !stop; ++it) {
                sl = slot_of<0>(plans, n_plans, sl, it);
                const TcnPlanDev& D = plans[sl];
                const long long local = it - D.item0;
                const long long t = local / D.items_per_tile;
                const int g = (int)(local - t * D.items_per_tile);
                const int u1 = min((g + 1) * D.upi, D.n_units);
                const unsigned bbytes = (unsigned)D.ns * kNK * 2u;
                const unsigned char* tb = D.bimg + (size_t)t * D.n_chunks * D.ns * 128;
                for (int u = g * D.upi; u < u1 && !stop; ++u) {
                    const TcnUnit U = D.units[u];
                    const unsigned abytes = (unsigned)U.abytes;
                    for (int kc = 0; kc < U.kchunks; ++kc, ++q) {
                        const int s = (int)(q % kNSlots);
                        const long long use = q / kNSlots;
                        if (s_abort || (use >= 1 && !bar_wait(&empty[s], (unsigned)((use - 1) & 1)))) {
                            abort_now(D.err);
                            stop = true;
                            break;
                        }
                        unsigned char* dst = ring + (size_t)s * kNSlotBytes;
                        const size_t asrc = 2 * (size_t)(U.a_off + (long long)kc * U.a_kstride);
                        const unsigned char* bsrc = tb + (size_t)(U.kc0 + kc) * D.ns * 128;
                        bar_expect(&full[s], split ? 2 * (abytes + bbytes) : abytes + bbytes);
                        bulk(dst, D.ahi + asrc, abytes, &full[s]);
                        bulk(dst + 2 * kNAHalf, bsrc, bbytes, &full[s]);
                        if (split) {
                            bulk(dst + kNAHalf, D.alo + asrc, abytes, &full[s]);
                            bulk(dst + 2 * kNAHalf + kNBHalf, bsrc + D.ns * 64, bbytes, &full[s]);
                        }
                        issued[s] = true;
                        par[s] = (unsigned)(use & 1);
                    }
                }
            }
            for (int s = 0; s < kNSlots; ++s)   // no copy left in flight
                if (issued[s]) bar_wait(&full[s], par[s]);
        }
    } else if (warp == kNWorkers + 1) {
        // ---------------- MMAs ----------------
        if (lane == 0) {
            long long q = 0;
            bool stop = false;
            int sl = slot0;
            for (long long it = i0, j = 0; it < i1 && !stop; ++it, ++j) {
                sl = slot_of<0>(plans, n_plans, sl, it);
                const TcnPlanDev& D = plans[sl];
                const int h = (int)(j & 1);
                const long long use_h = j >> 1;
                if (s_abort || (use_h >= 1 && !bar_wait(&acc_free[h], (unsigned)((use_h - 1) & 1)))) {
                    abort_now(D.err);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const long long local = it - D.item0;
                const long long t = local / D.items_per_tile;
                const int g = (int)(local - t * D.items_per_tile);
                const int u0 = g * D.upi, u1 = min(u0 + D.upi, D.n_units);
                const int ns = D.ns;
                const unsigned id = idesc(ns, !fp16);
                for (int u = u0; u < u1 && !stop; ++u) {
                    const TcnUnit U = D.units[u];
                    const int kmax = U.kmax;
                    const unsigned dt = tmem + (unsigned)(h * kNHalf + (u - u0) * ns);
                    for (int kc = 0; kc < U.kchunks; ++kc, ++q) {
                        const int s = (int)(q % kNSlots);
                        if (s_abort || !bar_wait(&full[s], (unsigned)((q / kNSlots) & 1))) {
                            abort_now(D.err);
                            stop = true;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const unsigned base = su32(ring + (size_t)s * kNSlotBytes);
                        const unsigned ahi = base, alo = base + kNAHalf;
                        const unsigned bhi = base + 2 * kNAHalf, blo = bhi + kNBHalf;
                        for (int ks = 0; ks < kNK / 16; ++ks) {
                            if (kc * kNK + ks * 16 >= kmax) break;
                            const unsigned koff = ks * 256u;
                            const unsigned long long ah = sdesc(ahi + koff, 128, 512);
                            const unsigned long long bh = sdesc(bhi + koff, 128, 512);
                            mma(dt, ah, bh, id, (kc | ks) ? 1u : 0u);
                            if (split) {
                                mma(dt, ah, sdesc(blo + koff, 128, 512), id, 1u);
                                mma(dt, sdesc(alo + koff, 128, 512), bh, id, 1u);
                            }
                        }
                        commit_to(&empty[s]);
                    }
                }
                if (!stop) commit_to(&acc_full[h]);
            }
            commit_to(&drain);             // arrives once every MMA issued above is complete
            bar_wait(&drain, 0);
        }
    } else {
        // ---------------- epilogue (warps 0-7) ----------------
        // warp w reads TMEM lanes 32 (w & 3) .. + 31; the two warps of a lane
        // quarter take alternate 16-column chunks.  An item's output
        // positions (cp.async) and signal scales are staged into the buffers
        // of its TMEM half while the item before it is stored.
        const int quarter = warp & 3, half16 = (warp >> 2) * 16;
        const unsigned lane_base = (unsigned)(quarter * 32) << 16;
        int sl = slot0, sl_st = slot0;
        auto stage = [&](long long it, int hh) {
            sl_st = slot_of<0>(plans, n_plans, sl_st, it);
            const TcnPlanDev& D = plans[sl_st];
            const long long local = it - D.item0;
            const long long t = local / D.items_per_tile;
            const int g = (int)(local - t * D.items_per_tile);
            const int u0 = g * D.upi, nu = min(u0 + D.upi, D.n_units) - u0;
            const int* src = D.upos + (size_t)u0 * kNM;
            for (int e = 4 * tid; e < nu * kNM; e += 4 * kNWorkers * 32)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(&s_pos[hh][e])), "l"(src + e)
                             : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
            const long long row0 = t * D.ns;
            const int rows = (int)min((long long)D.ns, D.batch - row0);
            if (tid < D.ns) s_sc[hh][tid] = (fp16 && tid < rows) ? D.scale[row0 + tid] : 1.f;   // tid < 256 covers ns <= 128
        };
        if (i0 < i1) stage(i0, 0);
        for (long long it = i0, j = 0; it < i1; ++it, ++j) {
            sl = slot_of<0>(plans, n_plans, sl, it);
            const TcnPlanDev& D = plans[sl];
            const int h = (int)(j & 1);
            const long long local = it - D.item0;
            const long long t = local / D.items_per_tile;
            const int g = (int)(local - t * D.items_per_tile);
            const int u0 = g * D.upi, u1 = min(u0 + D.upi, D.n_units);
            const int ns = D.ns, n = D.n;
            const long long row0 = t * ns;
            const int rows = (int)min((long long)ns, D.batch - row0);
            asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's staging of the item
            const bool bad = !bar_wait(&acc_full[h], (unsigned)((j >> 1) & 1));
            // the barrier also makes every thread's staging visible, and
            // every warp has finished the item before (the other half)
            if (workers_any(bad || s_abort != 0)) {
                if (tid == 0) abort_now(D.err);
                break;
            }
            if (it + 1 < i1) stage(it + 1, h ^ 1);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int u = u0; u < u1; ++u) {
                const int pos = s_pos[h][(u - u0) * kNM + quarter * 32 + lane];
                const bool valid = pos >= 0;
                for (int c0 = half16; c0 < ns; c0 += 32) {
                    unsigned r[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(tmem + lane_base + (unsigned)(h * kNHalf + (u - u0) * ns + c0)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (valid) {
#pragma unroll
                        for (int qq = 0; qq < 16; ++qq) {
                            const int s = c0 + qq;
                            if (s < rows) {
                                const float v = __uint_as_float(r[qq]) * s_sc[h][s];
                                __stcs(D.y + (row0 + s) * n + pos, v);
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(&acc_free[h]);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");   // no staging copy left in flight
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kNWorkers + 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kNCols) : "memory");
    }
}

}  // namespace
}  // namespace gft

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace gft {
namespace {

constexpr size_t kNSmemLimit = 232448;

struct TcnPlan {
    std::vector<TcnLeaf> leaves;
    TcnUnit* d_units = nullptr;         // per unit (M-tile of a leaf)
    int* d_upos = nullptr;              // per unit 128 output positions (-1 past the leaf's end)
    short* d_gather = nullptr;          // per chunk 32 node labels (-1: padding)
    int n_units = 0, n_chunks = 0;
    long long img_elems = 0;
    unsigned char* d_img[2][2] = {};   // [BF16, FP16][hi, lo]
    ~TcnPlan() {
        if (d_units) cudaFree(d_units);
        if (d_upos) cudaFree(d_upos);
        if (d_gather) cudaFree(d_gather);
        for (auto& a : d_img)
            for (auto& q : a)
                if (q) cudaFree(q);
    }
};

uint16_t bf16_of(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t r = ((u >> 16) & 1u) + 0x7FFFu;   // round to nearest even
    return (uint16_t)((u + r) >> 16);
}
float bf16_to_float(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

TcnPlan* tcn_prepare(gft_plan_s& p) {
    if (p.tcn) return static_cast<TcnPlan*>(p.tcn);
    std::unique_ptr<TcnPlan> T(new TcnPlan);
    int lab = 0, kc0 = 0, unit0 = 0;
    long long a = 0;
    std::vector<TcnUnit> units;
    std::vector<int> upos;
    for (size_t k = 0; k < p.leaves.size(); ++k) {
        const Leaf& lf = p.leaves[k];
        TcnLeaf L{};
        L.m = lf.m();
        L.npad = (L.m + 15) & ~15;
        L.kchunks = (L.m + kNK - 1) / kNK;
        L.mtiles = (L.npad + kNM - 1) / kNM;
        L.lab = lab;
        L.kc0 = kc0;
        L.unit0 = unit0;
        L.a_off = a;
        for (int mt = 0; mt < L.mtiles; ++mt) {
            TcnUnit U{};
            U.a_off = L.a_off + (long long)mt * kNM * kNK;
            U.a_kstride = L.npad * kNK;
            U.abytes = std::min(kNM, L.npad - mt * kNM) * kNK * 2;
            U.kchunks = L.kchunks;
            U.kc0 = L.kc0;
            U.kmax = (L.m + 15) & ~15;
            units.push_back(U);
            for (int r = 0; r < kNM; ++r) {
                const int c = mt * kNM + r;
                upos.push_back(c < L.m ? p.out_pos[(size_t)L.lab + c] : -1);
            }
        }
        lab += L.m;
        kc0 += L.kchunks;
        unit0 += L.mtiles;
        a += (long long)L.kchunks * L.npad * kNK;
        T->leaves.push_back(L);
    }
    T->n_units = unit0;
    T->n_chunks = kc0;
    std::vector<short> gat((size_t)kc0 * kNK, -1);
    for (size_t k = 0; k < p.leaves.size(); ++k) {
        const TcnLeaf& L = T->leaves[k];
        for (int r = 0; r < L.m; ++r) gat[(size_t)(L.kc0 + r / kNK) * kNK + r % kNK] = (short)p.leaves[k].labels[r];
    }
    GFT_CUDA(cudaMalloc(&T->d_gather, sizeof(short) * std::max<size_t>(1, gat.size())));
    GFT_CUDA(cudaMemcpy(T->d_gather, gat.data(), sizeof(short) * gat.size(), cudaMemcpyHostToDevice));
    T->img_elems = a;
    GFT_CUDA(cudaMalloc(&T->d_units, sizeof(TcnUnit) * units.size()));
    GFT_CUDA(cudaMemcpy(T->d_units, units.data(), sizeof(TcnUnit) * units.size(), cudaMemcpyHostToDevice));
    GFT_CUDA(cudaMalloc(&T->d_upos, sizeof(int) * upos.size()));
    GFT_CUDA(cudaMemcpy(T->d_upos, upos.data(), sizeof(int) * upos.size(), cudaMemcpyHostToDevice));
    p.tcn = T.release();
    return static_cast<TcnPlan*>(p.tcn);
}

// basis images of one precision: per leaf and 32-wide K chunk, npad rows
// (output coefficients c) x 32 K (inputs r) in the kernel's K-major
// core-matrix order; A[c][r] = M_k[r][c], split into hi and lo
void tcn_images(gft_plan_s& p, TcnPlan& T, bool fp16) {
    const int w = fp16 ? 1 : 0;
    if (T.d_img[w][0]) return;
    std::vector<uint16_t> hi((size_t)T.img_elems, 0), lo((size_t)T.img_elems, 0);
    for (size_t k = 0; k < p.leaves.size(); ++k) {
        const Leaf& lf = p.leaves[k];
        const TcnLeaf& L = T.leaves[k];
        for (int kc = 0; kc < L.kchunks; ++kc)
            for (int c = 0; c < L.m; ++c)
                for (int kk = 0; kk < kNK; ++kk) {
                    const int r = kc * kNK + kk;
                    if (r >= L.m) break;
                    const double val = lf.fold(r, c);
                    const size_t o = (size_t)L.a_off + (size_t)kc * L.npad * kNK +
                                     (size_t)(((c >> 3) * 4 + (kk >> 3)) * 64 + (c & 7) * 8 + (kk & 7));
                    if (fp16) {
                        const __half h = __float2half_rn((float)val);
                        hi[o] = __half_as_ushort(h);
                        lo[o] = __half_as_ushort(__float2half_rn((float)(val - (double)__half2float(h))));
                    } else {
                        const uint16_t h = bf16_of((float)val);
                        hi[o] = h;
                        lo[o] = bf16_of((float)(val - (double)bf16_to_float(h)));
                    }
                }
    }
    for (int q = 0; q < 2; ++q) {
        GFT_CUDA(cudaMalloc(&T.d_img[w][q], sizeof(uint16_t) * std::max<size_t>(1, hi.size())));
        GFT_CUDA(cudaMemcpy(T.d_img[w][q], (q ? lo : hi).data(), sizeof(uint16_t) * hi.size(), cudaMemcpyHostToDevice));
    }
}

int np_of(int n) { return ((n + 3) & ~3) + 4; }

struct TcnBatch {
    uint32_t prec = GFT_PREC_BF16X3;
    std::vector<int> members;            // slot -> index in the batch's plan list
    std::vector<TcnPlanDev> desc;
    TcnPlanDev* d_desc = nullptr;
    long long* d_range = nullptr;        // grid + 1 item boundaries
    int* d_first = nullptr;              // plan slot of each range's first item
    unsigned char* d_scratch = nullptr;  // B images and per-signal scales
    long long total_items = 0, total_groups = 0;
    int grid = 0;
    // pack launches: plans with short rows first (many warps per SM), then the rest
    long long pack_split = 0;
    int pack_grid[2] = {0, 0}, np_cap[2] = {4, 4};
    size_t pack_smem[2] = {0, 0};
    long long* d_pack_range[2] = {nullptr, nullptr};   // per part: grid + 1 group boundaries
    int* d_pack_first[2] = {nullptr, nullptr};
    ~TcnBatch() {
        for (void* q : {(void*)d_desc, (void*)d_range, (void*)d_first, (void*)d_scratch, (void*)d_pack_range[0],
                        (void*)d_pack_range[1], (void*)d_pack_first[0], (void*)d_pack_first[1]})
            if (q) cudaFree(q);
    }
};

}  // namespace

bool tcn_eligible(const gft_plan_s& p) {
    if (p.right || !p.has_device || p.n < 2) return false;
    for (auto& lf : p.leaves)
        if (lf.m() > kNMaxLeaf) return false;
    return (size_t)8 * np_of(p.n) * sizeof(float) + 2048 <= kNSmemLimit;
}

void tcn_free(gft_plan_s& p) {
    delete static_cast<TcnPlan*>(p.tcn);
    p.tcn = nullptr;
}

void* tcn_batch_create(const std::vector<gft_plan_s*>& plans, const std::vector<int64_t>& batches, uint32_t precision) {
    std::unique_ptr<TcnBatch> B(new TcnBatch);
    B->prec = precision;
    const bool fp16 = precision == GFT_PREC_FP16X3;
    const int k = (int)plans.size();
    std::vector<TcnPlanDev> d(k);
    std::vector<double> cost(k);          // per work item: bytes moved + a fixed cost
    for (int i = 0; i < k; ++i) {
        gft_plan_s& p = *plans[i];
        if (!tcn_eligible(p)) fail(GFT_ERR_UNSUPPORTED, "plan not supported by the few-signals tensor-core kernel");
        TcnPlan* T = tcn_prepare(p);
        tcn_images(p, *T, fp16);
        TcnPlanDev& e = d[i];
        e = TcnPlanDev{};
        e.batch = batches[i];
        e.prog = p.dev.d_ints;
        e.units = T->d_units;
        e.upos = T->d_upos;
        e.gather = T->d_gather;
        e.ahi = T->d_img[fp16 ? 1 : 0][0];
        e.alo = T->d_img[fp16 ? 1 : 0][1];
        e.err = p.dev.d_err;
        e.n = p.n;
        e.np = np_of(p.n);
        // signals per tile: the whole batch up to 128 (a multiple of 16)
        e.ns = (int)std::min<int64_t>(kNMaxNs, std::max<int64_t>(16, (batches[i] + 15) & ~int64_t(15)));
        e.n_units = T->n_units;
        e.n_chunks = T->n_chunks;
        e.n_stages = p.dev.n_pre_stages;
        e.n_pairs = p.dev.n_pairs;
        // units per item: one TMEM half, and at most kNItemSteps K chunks for
        // the widest leaf, so that a large graph spreads over many SMs and the
        // static ranges balance
        int kcmax = 1;
        for (auto& L : T->leaves) kcmax = std::max(kcmax, L.kchunks);
        e.upi = std::max(1, std::min({T->n_units, kNHalf / e.ns, kNItemSteps / kcmax}));
        e.items_per_tile = (T->n_units + e.upi - 1) / e.upi;
        double steps = 0;
        for (auto& L : T->leaves) steps += (double)L.mtiles * L.kchunks;
        cost[i] = steps / e.items_per_tile * (2.0 * kNAHalf + 2.0 * e.ns * kNK * 2) +
                  (double)e.upi * kNM * e.ns * 4.0 + 20000.0;
    }
    // slots: plans with rows of at most kPackShortNp floats first, each part
    // by decreasing cost per item
    auto part = [&](int i) { return d[i].np <= kPackShortNp ? 0 : 1; };
    B->members.resize(k);
    for (int i = 0; i < k; ++i) B->members[i] = i;
    std::stable_sort(B->members.begin(), B->members.end(), [&](int a, int b) {
        return part(a) != part(b) ? part(a) < part(b) : cost[a] > cost[b];
    });
    size_t scratch = 0;
    std::vector<size_t> off_img(k), off_scale(k);
    long long tiles_all = 0;
    for (int i : B->members) {
        TcnPlanDev e = d[i];
        const long long tiles = (e.batch + e.ns - 1) / e.ns;
        e.tile0 = tiles_all;
        e.item0 = B->total_items;
        e.grp0 = B->total_groups;
        tiles_all += tiles;
        B->total_items += tiles * e.items_per_tile;
        B->total_groups += tiles * (e.ns / 8);
        if (part(i) == 0) B->pack_split = B->total_groups;
        B->np_cap[part(i)] = std::max(B->np_cap[part(i)], e.np);
        off_img[i] = scratch;
        scratch += (size_t)tiles * e.n_chunks * e.ns * 128;
        scratch = (scratch + 255) & ~size_t(255);
        off_scale[i] = scratch;
        scratch += sizeof(float) * (size_t)tiles * e.ns;
        scratch = (scratch + 255) & ~size_t(255);
        B->desc.push_back(e);
    }
    GFT_CUDA(cudaMalloc(&B->d_scratch, std::max<size_t>(scratch, 256)));
    for (size_t sl = 0; sl < B->desc.size(); ++sl) {
        const int i = B->members[sl];
        B->desc[sl].bimg = B->d_scratch + off_img[i];
        B->desc[sl].scale = reinterpret_cast<float*>(B->d_scratch + off_scale[i]);
    }
    // main kernel: one CTA per SM, contiguous item ranges of about equal cost
    const size_t smem = (size_t)kNSlots * kNSlotBytes;
    GFT_CUDA(cudaFuncSetAttribute(tcn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    B->grid = (int)std::max<long long>(1, std::min<long long>(B->total_items, sm_count()));
    double total = 0.0;
    for (size_t sl = 0; sl < B->desc.size(); ++sl) {
        const TcnPlanDev& e = B->desc[sl];
        total += cost[B->members[sl]] * (double)((e.batch + e.ns - 1) / e.ns * e.items_per_tile);
    }
    std::vector<long long> range(B->grid + 1, B->total_items);
    std::vector<int> first(B->grid, std::max(0, (int)B->desc.size() - 1));
    range[0] = 0;
    first[0] = 0;
    double acc = 0.0;
    int cta = 1;
    for (size_t sl = 0; sl < B->desc.size() && cta < B->grid; ++sl) {
        const TcnPlanDev& e = B->desc[sl];
        const long long items = (e.batch + e.ns - 1) / e.ns * e.items_per_tile;
        for (long long t = 0; t < items && cta < B->grid; ++t) {
            acc += cost[B->members[sl]];
            while (cta < B->grid && acc >= total * cta / B->grid) {
                range[cta] = std::min(e.item0 + t + 1, B->total_items);
                first[cta] = (int)sl;
                ++cta;
            }
        }
    }
    // pack kernels: contiguous group ranges of about equal cost (row length
    // plus a fixed cost) per CTA, in each part
    GFT_CUDA(cudaFuncSetAttribute(tcn_pack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kNSmemLimit - 1024)));
    for (int c = 0; c < 2; ++c) {
        const long long g0 = c == 0 ? 0 : B->pack_split, g1 = c == 0 ? B->pack_split : B->total_groups;
        B->pack_smem[c] = (size_t)8 * B->np_cap[c] * sizeof(float);
        int per_sm = 0;
        GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tcn_pack_kernel, kPackThreads, B->pack_smem[c]));
        per_sm = std::max(1, per_sm);
        const int grid = (int)std::max<long long>(0, std::min<long long>(g1 - g0, (long long)per_sm * sm_count()));
        B->pack_grid[c] = grid;
        if (!grid) continue;
        double tot = 0.0;
        for (const TcnPlanDev& e : B->desc)
            if (e.grp0 >= g0 && e.grp0 < g1) tot += (double)((e.batch + e.ns - 1) / e.ns * (e.ns / 8)) * (e.n + 64.0);
        std::vector<long long> pr(grid + 1, g1);
        std::vector<int> pf(grid, 0);
        pr[0] = g0;
        int first_sl = 0;
        while (first_sl + 1 < (int)B->desc.size() && B->desc[first_sl + 1].grp0 <= g0) ++first_sl;
        pf[0] = first_sl;
        for (int b = 1; b < grid; ++b) pf[b] = (int)B->desc.size() - 1;
        double acc = 0.0;
        int cta = 1;
        for (size_t sl = first_sl; sl < B->desc.size() && cta < grid; ++sl) {
            const TcnPlanDev& e = B->desc[sl];
            if (e.grp0 >= g1) break;
            const long long groups = (e.batch + e.ns - 1) / e.ns * (e.ns / 8);
            for (long long q = 0; q < groups && cta < grid; ++q) {
                acc += e.n + 64.0;
                while (cta < grid && acc >= tot * cta / grid) {
                    pr[cta] = e.grp0 + q + 1;
                    pf[cta] = (int)sl;
                    ++cta;
                }
            }
        }
        GFT_CUDA(cudaMalloc(&B->d_pack_range[c], sizeof(long long) * pr.size()));
        GFT_CUDA(cudaMalloc(&B->d_pack_first[c], sizeof(int) * pf.size()));
        GFT_CUDA(cudaMemcpy(B->d_pack_range[c], pr.data(), sizeof(long long) * pr.size(), cudaMemcpyHostToDevice));
        GFT_CUDA(cudaMemcpy(B->d_pack_first[c], pf.data(), sizeof(int) * pf.size(), cudaMemcpyHostToDevice));
    }
    GFT_CUDA(cudaMalloc(&B->d_desc, sizeof(TcnPlanDev) * std::max<size_t>(1, B->desc.size())));
    GFT_CUDA(cudaMalloc(&B->d_range, sizeof(long long) * range.size()));
    GFT_CUDA(cudaMalloc(&B->d_first, sizeof(int) * first.size()));
    GFT_CUDA(cudaMemcpy(B->d_range, range.data(), sizeof(long long) * range.size(), cudaMemcpyHostToDevice));
    GFT_CUDA(cudaMemcpy(B->d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
    return B.release();
}

void tcn_batch_upload(void* h, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st) {
    TcnBatch* B = static_cast<TcnBatch*>(h);
    for (size_t sl = 0; sl < B->desc.size(); ++sl) {
        B->desc[sl].x = x[B->members[sl]];
        B->desc[sl].y = y[B->members[sl]];
    }
    if (!B->desc.empty())
        GFT_CUDA(cudaMemcpyAsync(B->d_desc, B->desc.data(), sizeof(TcnPlanDev) * B->desc.size(), cudaMemcpyHostToDevice,
                                 st));
}

void tcn_batch_launch(void* h, cudaStream_t st) {
    TcnBatch* B = static_cast<TcnBatch*>(h);
    if (B->total_items == 0) return;
    for (int c = 0; c < 2; ++c) {
        if (B->pack_grid[c] == 0) continue;
        tcn_pack_kernel<<<B->pack_grid[c], kPackThreads, B->pack_smem[c], st>>>(
            B->d_desc, (int)B->desc.size(), B->d_pack_range[c], B->d_pack_first[c], (int)B->prec);
        GFT_CUDA(cudaGetLastError());
    }
    tcn_kernel<<<B->grid, kNThreads, (size_t)kNSlots * kNSlotBytes, st>>>(B->d_desc, (int)B->desc.size(), B->d_range,
                                                                         B->d_first, (int)B->prec);
    GFT_CUDA(cudaGetLastError());
}

void tcn_batch_free(void* h) { delete static_cast<TcnBatch*>(h); }

int tcn_batch_launches(void* h) {
    const TcnBatch* B = static_cast<TcnBatch*>(h);
    if (B->total_items == 0) return 0;
    return 1 + (B->pack_grid[0] > 0 ? 1 : 0) + (B->pack_grid[1] > 0 ? 1 : 0);
}

}  // namespace gft

// Leaf products on the 5th-generation tensor cores (tcgen05, TMEM).
//
// For leaves too large for the CUDA-core kernels (m > 64: the 16x16 and
// 32x32 grids, the 256-cycle, large bipartite graphs) the leaf products
// y_k = M_k^T v_k (Sec. IV-C, Eq. 13; M_k the folded leaf basis) are dense
// contractions, run here as GEMMs D[128 x N] = A[128 x K] B[K x N] per tile
// of 128 signals:
//   1. tc_pack8_kernel: eight signals per warp step, staged in shared
//      memory by cp.async; the Haar stages in place; each post-stage value
//      converted to BF16 (hi, and lo = v - hi for the split precisions) or
//      per-signal scaled FP16 hi/lo, and written as ready-made shared-memory
//      images: per tile of 128 signals and per item (leaf, K chunk of 64), a
//      128 x 64 block in the canonical no-swizzle K-major layout (8 x 16-byte
//      core matrices), hi then lo, with 512-byte coalesced stores;
//   2. tc_leaf_kernel (persistent, one CTA per SM, warp-specialised): a
//      copy thread streams the A images (and B images unless they are
//      resident) through a ring of shared-memory slots with bulk copies, an
//      MMA thread issues tcgen05.mma (M=128, N=leaf width, K=16 per
//      instruction) into the leaf's TMEM columns -- one product for BF16,
//      three (hi*hi + hi*lo + lo*hi) for the split precisions -- and eight
//      epilogue warps read the double-buffered accumulators (groups of
//      leaves of at most 256 columns) column by column IN COEFFICIENT ORDER
//      (tcgen05.ld 32x32b), so the ascending-eigenvalue permutation costs
//      nothing, and store 32 output positions per row.  Every wait is bounded
//      (about 2 s, then GFT_ERR_TIMEOUT, drain, TMEM freed).
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

constexpr int kTcM = 128;        // signals per tile = MMA M
constexpr int kTcK = 64;         // K chunk staged per step
constexpr int kTcThreads = 320;  // warps 0-7 epilogue (two per 32-lane TMEM quarter), 8 copies, 9 MMAs
constexpr int kTcEpiWarps = 8;
constexpr int kTcMaxN = 256;     // widest leaf handled in one MMA
constexpr int kTcCols = 512;     // TMEM columns allocated per CTA (one CTA per SM)
constexpr int kTcGroupCols = 256;   // columns of one accumulator buffer (two buffers)

struct TcLeaf {
    int m;        // leaf size
    int npad;     // N padded to a multiple of 16
    int kchunks;  // ceil(m / 64)
    int off;      // offset in leaf-concatenated order
    int tcol;     // TMEM column of this leaf's first output (within its group)
    int group;
    long long b_off;  // element offset of the leaf's B image (per precision array)
};

struct TcItem;
// One plan of a launch (a launch may cover many plans: mixed batches).
struct TcPlanDev {
    const float* x;              // [batch, n] signals
    float* y;                    // [batch, n] coefficients
    unsigned char* aimg;         // split operand images, [tiles][items] x 32 KB
    float* scale;                // per-signal FP16 scale
    long long batch;
    long long tile0, group0;     // first tile / first 8-signal group of this plan in the launch
    const TcItem* items;
    const TcLeaf* leaves;
    const int* gmap;             // [2n + 2(G+1)]: per leaf group (outputs sorted): coefficient index,
                                 // TMEM column; then group offsets, then the first item of each group
    const short* gather;         // [items][64]: slot feeding each K index (-1: padding)
    const int* prog;             // the plan's program head: [pairs 2P][stage offsets S+1]
    const unsigned char* bhi;    // pre-split B images in this launch's format: hi, lo
    const unsigned char* blo;
    int n, n_items, n_leaves, n_groups, n_pairs, n_stages;
    unsigned total_b;            // bytes of all hi B images (resident mode)
};

// plan of launch-wide index `v` (first-index array: tile0 or group0)
template <bool TILES>
__device__ __forceinline__ int find_plan(const TcPlanDev* P, int n_plans, long long v) {
    int lo = 0, hi = n_plans - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((TILES ? P[mid].tile0 : P[mid].group0) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, canonical K-major layout without swizzle:
// start >> 4 in bits 0-13, leading-dimension byte offset (between core
// matrices adjacent along K) >> 4 in bits 16-29, stride byte offset (between
// 8-row groups) >> 4 in bits 32-45, descriptor version 1 in bits 46-47,
// swizzle mode 0 in bits 61-63
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// instruction descriptor for kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B format (bits 7-9, 10-12: 1 = BF16, 0 = FP16), both K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ __forceinline__ unsigned instr_desc(int n, bool bf16) {
    unsigned d = 0;
    d |= 1u << 4;
    if (bf16) d |= (1u << 7) | (1u << 10);
    d |= (unsigned)((n >> 3) & 0x3F) << 17;
    d |= (unsigned)((kTcM >> 4) & 0x1F) << 24;
    return d;
}

__device__ __forceinline__ void mma_f16(unsigned dt, unsigned long long ad, unsigned long long bd, unsigned id,
                                        unsigned acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mbar_init1(unsigned long long* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try1(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok)
                 : "r"(smem_u32(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* b, unsigned parity) {
    if (mbar_try1(b, parity)) return true;
    const unsigned long long t0 = gtimer_ns();
    while (!mbar_try1(b, parity))
        if (gtimer_ns() - t0 > 2000000000ull) return false;
    return true;
}

// one 16-byte row of a core matrix: byte offset of (row, k-group) in a
// [rows x 64] K-major no-swizzle tile whose 8-row groups are 1024 B apart
__device__ __forceinline__ unsigned core_off(int row, int kg) {
    return (unsigned)(((row >> 3) * 8 + kg) * 128 + (row & 7) * 16);
}

__device__ __forceinline__ void mbar_expect(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}

// Work item = (leaf, K chunk); items of a tile run in leaf order.
struct TcItem {
    int leaf, kc;
    int bres;   // byte offset of this item's B image among the resident images (hi set)
};

// Persistent tensor-core kernel, one CTA per SM, warp-specialised:
//   warp 8 (one thread) bulk-loads (TMA) the A image of each work item
//     (leaf, 64-wide K chunk) of each tile -- written by tc_pack8_kernel --
//     and, unless every B image is resident, the item's B images, into a
//     ring of shared-memory slots (4 slots of A when all B images fit in
//     96 KB and are loaded once, else 2 slots of A + B);
//   warp 9 (one thread) waits for a slot, issues its MMAs (M = 128 signals,
//     N = leaf width, K = 16 per instruction; one product for BF16, three
//     -- hi*hi + hi*lo + lo*hi -- for the split precisions) into the TMEM
//     columns of the item's leaf, and commits them to the slot's "empty"
//     barrier; after the last item of a leaf group it commits to the group's
//     "accumulator full" barrier;
//   warps 0-7 (the epilogue; warp w reads TMEM lanes 32 (w & 3) .. + 31, the
//     two warps of a lane quarter take alternate 16-column chunks) wait for
//     a full accumulator, read its columns in coefficient order, transpose
//     32 x 16 blocks through shared memory and store 16 consecutive output
//     positions of two rows per instruction, then release the accumulator.
// Leaves are grouped so that a group needs at most 256 TMEM columns; the
// accumulator is double buffered (2 x 256 of the 512 columns), so the
// epilogue of one group overlaps the copies and MMAs of the next.  When all
// leaves form one group the stores are 128-byte row segments in output
// order; otherwise each group writes its own (sorted) output positions.
// Every wait gives up after about two seconds (GFT_ERR_TIMEOUT in the plan's
// error word; all roles leave their loops; copies and MMAs in flight are
// awaited, again bounded, before the TMEM columns are freed).
struct TcRing {
    int resident;       // B images resident in shared memory (single-plan launches only)
    int nbuf;           // ring depth
    unsigned bufsz;     // bytes per ring buffer
    unsigned bslot;     // streamed mode: byte offset of the B images inside a ring buffer
    unsigned res_off;   // resident mode: byte offset of the resident B region
    unsigned stage_off; // byte offset of the epilogue staging
    unsigned meta_off;  // single-plan launches: byte offset of [items][leaves][gmap]
};

constexpr int kStageLd = 17;   // epilogue staging row stride (floats): 16 columns + 1, conflict-free

// Work units are the tiles of every plan of the launch, in plan order; CTA b
// takes units b, b + grid, ... (every role walks the same sequence).
__global__ void __launch_bounds__(kTcThreads, 1) tc_leaf_kernel(TcPlanDev one, const TcPlanDev* __restrict__ many,
                                                               int n_plans, long long total_tiles, int prec,
                                                               int* err, TcRing ring) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ unsigned s_tmem;
    __shared__ __align__(8) unsigned long long bar_full[4], bar_empty[4], bar_dfull[2], bar_dfree[2], bar_b;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* s_stage = reinterpret_cast<float*>(sm + ring.stage_off);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) {
            mbar_init1(&bar_full[i]);
            mbar_init1(&bar_empty[i]);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init1(&bar_dfull[i]);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_dfree[i])), "r"(kTcEpiWarps)
                         : "memory");
        }
        mbar_init1(&bar_b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    const bool split = prec != GFT_PREC_BF16;
    const bool fp16 = prec == GFT_PREC_FP16X3;
    const unsigned a_bytes = split ? 32768u : 16384u;
    const long long my_units = total_tiles > blockIdx.x ? (total_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    unsigned char* res = sm + ring.res_off;
    // a single-plan launch reads its tables from shared-memory copies
    const TcItem* l_items = one.items;
    const TcLeaf* l_leaves = one.leaves;
    const int* l_gmap = one.gmap;
    if (!many) {
        unsigned char* meta = sm + ring.meta_off;
        TcItem* s_items = reinterpret_cast<TcItem*>(meta);
        const size_t items_bytes = (sizeof(TcItem) * one.n_items + 15) & ~size_t(15);
        TcLeaf* s_leaves = reinterpret_cast<TcLeaf*>(meta + items_bytes);
        const size_t leaves_bytes = (sizeof(TcLeaf) * one.n_leaves + 15) & ~size_t(15);
        int* s_gmap = reinterpret_cast<int*>(meta + items_bytes + leaves_bytes);
        const int gmap_ints = 2 * one.n + 2 * (one.n_groups + 1);
        for (int i = tid; i < one.n_items; i += blockDim.x) s_items[i] = one.items[i];
        for (int i = tid; i < one.n_leaves; i += blockDim.x) s_leaves[i] = one.leaves[i];
        for (int i = tid; i < gmap_ints; i += blockDim.x) s_gmap[i] = one.gmap[i];
        l_items = s_items;
        l_leaves = s_leaves;
        l_gmap = s_gmap;
        __syncthreads();
    }
    auto plan_of = [&](long long t, long long& tile) -> TcPlanDev {
        if (!many) {
            tile = t;
            TcPlanDev D = one;
            D.items = l_items;
            D.leaves = l_leaves;
            D.gmap = l_gmap;
            return D;
        }
        const int p = find_plan<true>(many, n_plans, t);
        tile = t - many[p].tile0;
        return many[p];
    };
    auto abort_now = [&]() {
        s_abort = 1;
        atomicExch(err, (int)GFT_ERR_TIMEOUT);
    };

    if (warp == kTcEpiWarps) {
        // ---------------- copies ----------------
        if (lane == 0) {
            if (ring.resident && my_units > 0) {
                mbar_expect(&bar_b, split ? 2 * one.total_b : one.total_b);
                for (int i = 0; i < one.n_items; ++i) {
                    const TcItem it = l_items[i];
                    const TcLeaf L = l_leaves[it.leaf];
                    const unsigned b_bytes = (unsigned)L.npad * kTcK * 2u;
                    const size_t src = 2 * (size_t)(L.b_off + (long long)it.kc * L.npad * kTcK);
                    bulk_load(res + it.bres, one.bhi + src, b_bytes, &bar_b);
                    if (split) bulk_load(res + one.total_b + it.bres, one.blo + src, b_bytes, &bar_b);
                }
            }
            long long q = 0;
            bool issued[4] = {false, false, false, false};
            unsigned last_par[4] = {0, 0, 0, 0};
            for (long long k = 0; k < my_units && !s_abort; ++k) {
                long long tile;
                const TcPlanDev D = plan_of(blockIdx.x + k * (long long)gridDim.x, tile);
                for (int i = 0; i < D.n_items && !s_abort; ++i, ++q) {
                    const int s = (int)(q % ring.nbuf);
                    if (q >= ring.nbuf && !mbar_wait_bounded(&bar_empty[s], (unsigned)(((q / ring.nbuf) - 1) & 1))) {
                        abort_now();
                        break;
                    }
                    const TcItem it = D.items[i];
                    const TcLeaf L = D.leaves[it.leaf];
                    unsigned char* b = sm + (size_t)s * ring.bufsz;
                    const unsigned b_bytes = (unsigned)L.npad * kTcK * 2u;
                    mbar_expect(&bar_full[s], a_bytes + (ring.resident ? 0u : (split ? 2 * b_bytes : b_bytes)));
                    bulk_load(b, D.aimg + ((size_t)tile * D.n_items + (size_t)i) * 32768u, a_bytes, &bar_full[s]);
                    if (!ring.resident) {
                        const size_t src = 2 * (size_t)(L.b_off + (long long)it.kc * L.npad * kTcK);
                        bulk_load(b + ring.bslot, D.bhi + src, b_bytes, &bar_full[s]);
                        if (split) bulk_load(b + ring.bslot + b_bytes, D.blo + src, b_bytes, &bar_full[s]);
                    }
                    issued[s] = true;
                    last_par[s] = (unsigned)((q / ring.nbuf) & 1);
                }
            }
            for (int s = 0; s < 4; ++s)   // no copy left in flight
                if (issued[s]) mbar_wait_bounded(&bar_full[s], last_par[s]);
            if (ring.resident && my_units > 0) mbar_wait_bounded(&bar_b, 0);
        }
    } else if (warp == kTcEpiWarps + 1) {
        // ---------------- MMAs ----------------
        if (lane == 0) {
            if (ring.resident && my_units > 0 && !mbar_wait_bounded(&bar_b, 0)) abort_now();
            long long q = 0, u = 0;
            bool pending = false;
            for (long long k = 0; k < my_units && !s_abort; ++k) {
                long long tile;
                const TcPlanDev D = plan_of(blockIdx.x + k * (long long)gridDim.x, tile);
                for (int g = 0; g < D.n_groups && !s_abort; ++g, ++u) {
                    const int buf = (int)(u & 1);
                    if (u >= 2 && !mbar_wait_bounded(&bar_dfree[buf], (unsigned)(((u >> 1) - 1) & 1))) {
                        abort_now();
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int* gitem = D.gmap + 2 * D.n + D.n_groups + 1;
                    for (int i = gitem[g]; i < gitem[g + 1]; ++i, ++q) {
                        const int s = (int)(q % ring.nbuf);
                        if (!mbar_wait_bounded(&bar_full[s], (unsigned)((q / ring.nbuf) & 1))) {
                            abort_now();
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const TcItem it = D.items[i];
                        const TcLeaf L = D.leaves[it.leaf];
                        const unsigned id = instr_desc(L.npad, !fp16);
                        const unsigned dt = tmem + (unsigned)(buf * kTcGroupCols + L.tcol);
                        const unsigned abase = smem_u32(sm + (size_t)s * ring.bufsz);
                        const unsigned b_bytes = (unsigned)L.npad * kTcK * 2u;
                        const unsigned bhi = ring.resident ? smem_u32(res + it.bres) : abase + ring.bslot;
                        const unsigned blo = ring.resident ? smem_u32(res + D.total_b + it.bres) : bhi + b_bytes;
                        for (int ks = 0; ks < kTcK / 16; ++ks) {
                            if (it.kc * kTcK + ks * 16 >= ((L.m + 15) & ~15)) break;
                            const unsigned koff = ks * 256u;
                            const unsigned long long ah = smem_desc(abase + koff, 128, 1024);
                            const unsigned long long bh = smem_desc(bhi + koff, 128, 1024);
                            mma_f16(dt, ah, bh, id, (it.kc | ks) ? 1u : 0u);
                            if (split) {
                                mma_f16(dt, ah, smem_desc(blo + koff, 128, 1024), id, 1u);
                                mma_f16(dt, smem_desc(abase + 16384u + koff, 128, 1024), bh, id, 1u);
                            }
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                         smem_u32(&bar_empty[s]))
                                     : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&bar_dfull[buf]))
                                 : "memory");
                    pending = true;
                }
            }
            if (pending) {   // every MMA done before the columns are freed
                const long long last = u - 1;
                mbar_wait_bounded(&bar_dfull[(int)(last & 1)], (unsigned)((last >> 1) & 1));
            }
        }
    } else {
        // ---------------- epilogue (warps 0-7) ----------------
        // warp w reads TMEM lanes 32 (w & 3) .. + 31 (its quarter); the two
        // warps of a quarter take alternate 16-column chunks
        const int quarter = warp & 3, half = warp >> 2;
        float* stg = s_stage + warp * 32 * kStageLd;
        const unsigned lane_base = (unsigned)(quarter * 32) << 16;
        long long u = 0;
        for (long long k = 0; k < my_units && !s_abort; ++k) {
            long long tile;
            const TcPlanDev D = plan_of(blockIdx.x + k * (long long)gridDim.x, tile);
            const long long r0 = tile * kTcM + quarter * 32;
            const long long row = r0 + lane;
            const float sc = fp16 ? (row < D.batch ? D.scale[row] : 1.f) : 1.f;
            const int* gpos = D.gmap;
            const int* gcol = D.gmap + D.n;
            const int* goff = D.gmap + 2 * D.n;
            for (int g = 0; g < D.n_groups && !s_abort; ++g, ++u) {
                const int buf = (int)(u & 1);
                if (!mbar_wait_bounded(&bar_dfull[buf], (unsigned)((u >> 1) & 1))) {
                    if (lane == 0) abort_now();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int j_end = goff[g + 1];
                for (int j0 = goff[g] + 16 * half; j0 < j_end; j0 += 32) {
                    const int cnt = min(16, j_end - j0);
                    const int c = lane & 15;
                    const int my_col = c < cnt ? gcol[j0 + c] : gcol[j_end - 1];
                    const int pos = c < cnt ? gpos[j0 + c] : 0;
                    float r[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int col = __shfl_sync(0xffffffffu, my_col, q);
                        unsigned uu;
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                                     : "=r"(uu)
                                     : "r"(tmem + lane_base + (unsigned)(buf * kTcGroupCols + col)));
                        r[q] = __uint_as_float(uu);
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    // transpose through shared memory: lane = row -> (row pair, output position)
#pragma unroll
                    for (int q = 0; q < 16; ++q) stg[lane * kStageLd + q] = r[q] * sc;
                    __syncwarp();
#pragma unroll 4
                    for (int rr = 0; rr < 16; ++rr) {
                        const int rl = 2 * rr + (lane >> 4);
                        const long long grow = r0 + rl;
                        if (grow < D.batch && c < cnt) __stcs(D.y + grow * D.n + pos, stg[rl * kStageLd + c]);
                    }
                    __syncwarp();
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_dfree[buf])) : "memory");
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}

// A images, eight signals per warp step.  A warp owns a group of 8
// consecutive signals (one 8-row block of the core-matrix layout): the rows
// arrive in a per-warp shared buffer (row stride n + 4) by 16-byte cp.async
// copies, the next group's copies overlapping this group's work; the Haar
// units of every stage run in place; for FP16 the warp also computes each
// signal's power-of-two scale (written to `scale`).  Lane (r, sub) then
// forms 16-byte core-matrix rows for K groups kg = sub, sub + 4, ...: the 32
// lanes of a store instruction cover 4 K groups x 8 rows = 512 contiguous
// bytes of the image, hi and lo.  gather[item * 64 + k] is the slot whose
// value feeds K index k of the item (-1: zero padding).
constexpr int kPack8Warps = 4;

// Copies of the 8 rows starting at row0 of plan D into a warp's staging
// buffer (row stride rs), one commit group.
__device__ __forceinline__ void pack_issue(const TcPlanDev& D, long long row0, float* buf, int rs, int lane) {
    const int n = D.n;
    const int valid = (int)max(0LL, min(8LL, D.batch - row0));
    if ((n & 3) == 0) {
        const int per = n >> 2;
        for (int c = lane; c < valid * per; c += 32) {
            const int r = c / per, kk = c - r * per;
            const unsigned d = (unsigned)__cvta_generic_to_shared(buf + r * rs + 4 * kk);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(D.x + (row0 + r) * n + 4 * kk)
                         : "memory");
        }
    } else {
        for (int c = lane; c < valid * n; c += 32) {
            const int r = c / n, kk = c - r * n;
            const unsigned d = (unsigned)__cvta_generic_to_shared(buf + r * rs + kk);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(D.x + (row0 + r) * n + kk) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// One group of 8 signals (rows row0.. of plan D, rows rt.. of tile `tile`)
// already in the warp's buffer: FP16 scales, Haar units in place, split
// operand rows stored.  s_pairs / s_soff / s_gather: the plan's tables.
__device__ __forceinline__ void pack_group(const TcPlanDev& D, float* buf, int rs, long long row0, long long tile,
                                           int rt, const int* s_pairs, const int* s_soff, const short* s_gather,
                                           bool fp16, bool split, int lane) {
    const int n = D.n;
    const int valid = (int)max(0LL, min(8LL, D.batch - row0));
    float inv[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) inv[r] = 1.f;
    if (fp16) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            float m = 0.f;
            if (r < valid)
                for (int c = lane; c < n; c += 32) m = fmaxf(m, fabsf(buf[r * rs + c]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            const float sc = m > 0.f ? exp2f(ceilf(log2f(m)) + (float)D.n_stages) : 1.f;
            inv[r] = 1.f / sc;
            if (lane == 0 && r < valid) D.scale[row0 + r] = sc;
        }
    }
    // Haar units: lanes over the pairs of a stage, the 8 rows unrolled (rows
    // past the batch hold stale values that are never stored)
    for (int s = 0; s < D.n_stages; ++s) {
        const int p1 = s_soff[s + 1];
        for (int pp = s_soff[s] + lane; pp < p1; pp += 32) {
            const int2 uv = *reinterpret_cast<const int2*>(s_pairs + 2 * pp);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                float* row = buf + r * rs;
                const float xu = row[uv.x], xv = row[uv.y];
                row[uv.x] = xu + xv;
                row[uv.y] = xu - xv;
            }
        }
        __syncwarp();
    }
    const int r = lane & 7, sub = lane >> 3;
    const bool live = r < valid;
    const float* row = buf + r * rs;
    const float sc = inv[r];
    for (int kg = sub; kg < D.n_items * 8; kg += 4) {
        float v[8];
        const int4 g4 = *reinterpret_cast<const int4*>(s_gather + kg * 8);   // eight slot indices
        const short* gs = reinterpret_cast<const short*>(&g4);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int lab = gs[e];
            v[e] = (live && lab >= 0) ? row[lab] * sc : 0.f;
        }
        unsigned hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {   // two values per conversion instruction
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
        const int item = kg >> 3;
        unsigned char* dst = D.aimg + ((size_t)tile * D.n_items + item) * 32768u + core_off(rt + r, kg & 7);
        __stcg(reinterpret_cast<uint4*>(dst), make_uint4(hi[0], hi[1], hi[2], hi[3]));
        if (split) __stcg(reinterpret_cast<uint4*>(dst + 16384), make_uint4(lo[0], lo[1], lo[2], lo[3]));
    }
    __syncwarp();   // buffer reusable by the copies issued next
}

// One plan: every warp walks groups G = blockIdx.x * W + warp + k * (grid * W)
// (consecutive groups on consecutive warps), prefetching its next group
// while it packs the current one; the tables are loaded once.
__global__ void __launch_bounds__(kPack8Warps * 32) tc_pack8_kernel(TcPlanDev D, int rs, int nbuf, int prec) {
    extern __shared__ __align__(16) float sbuf[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* wbuf = sbuf + (size_t)warp * nbuf * 8 * rs;
    const int prog_ints = 2 * D.n_pairs + D.n_stages + 1;
    int* s_prog = reinterpret_cast<int*>(sbuf + (size_t)kPack8Warps * nbuf * 8 * rs);
    short* s_gather = reinterpret_cast<short*>(s_prog + ((prog_ints + 3) & ~3));   // 16-byte aligned
    for (int i = tid; i < prog_ints; i += blockDim.x) s_prog[i] = D.prog[i];
    for (int i = tid; i < D.n_items * 64; i += blockDim.x) s_gather[i] = D.gather[i];
    __syncthreads();
    const bool fp16 = prec == GFT_PREC_FP16X3, split = prec != GFT_PREC_BF16;
    const long long n_groups = (D.batch + kTcM - 1) / kTcM * (kTcM / 8);
    const long long stride = (long long)gridDim.x * kPack8Warps;
    long long G = blockIdx.x * (long long)kPack8Warps + warp;
    int cur = 0;
    if (G < n_groups) pack_issue(D, G * 8, wbuf, rs, lane);
    for (; G < n_groups; G += stride) {
        float* buf = wbuf + cur * 8 * rs;
        const bool has_next = G + stride < n_groups;
        if (nbuf == 2 && has_next) pack_issue(D, (G + stride) * 8, wbuf + (cur ^ 1) * 8 * rs, rs, lane);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncwarp();
        const long long row0 = G * 8;
        const long long tile = row0 / kTcM;
        pack_group(D, buf, rs, row0, tile, (int)(row0 - tile * kTcM), s_prog, s_prog + 2 * D.n_pairs, s_gather, fp16,
                   split, lane);
        if (nbuf == 2) cur ^= 1;
        else if (has_next) pack_issue(D, (G + stride) * 8, wbuf, rs, lane);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Many plans (mixed batches): work units are the tiles of every plan (in
// plan order); CTA b takes tiles b, b + grid, ...; warp w packs groups w,
// w+4, w+8, w+12 of each tile.  A plan's tables are loaded into shared
// memory when the next tile belongs to another plan.
__global__ void __launch_bounds__(kPack8Warps * 32) tc_pack8_multi_kernel(const TcPlanDev* __restrict__ many,
                                                                          int n_plans, long long total_tiles, int rs,
                                                                          int prog_cap, int prec, int nbuf) {
    extern __shared__ __align__(16) float sbuf[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* wbuf = sbuf + (size_t)warp * nbuf * 8 * rs;
    int* s_prog = reinterpret_cast<int*>(sbuf + (size_t)kPack8Warps * nbuf * 8 * rs);
    short* s_gather = reinterpret_cast<short*>(s_prog + ((prog_cap + 3) & ~3));   // 16-byte aligned
    const bool fp16 = prec == GFT_PREC_FP16X3, split = prec != GFT_PREC_BF16;
    const long long my_units = total_tiles > blockIdx.x ? (total_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    constexpr int kPer = kTcM / 8 / kPack8Warps;   // groups per warp per tile
    // rows of step (k, j): tile blockIdx.x + k * grid, group kPack8Warps * j + warp
    auto step_row0 = [&](long long k, int j, int& p) -> long long {
        const long long t = blockIdx.x + k * (long long)gridDim.x;
        p = find_plan<true>(many, n_plans, t);
        return (t - many[p].tile0) * kTcM + (long long)(kPack8Warps * j + warp) * 8;
    };
    int loaded = -1, cur = 0;
    if (my_units > 0) {
        int p0;
        const long long r0 = step_row0(0, 0, p0);
        pack_issue(many[p0], r0, wbuf, rs, lane);
    }
    for (long long k = 0; k < my_units; ++k) {
        int p;
        step_row0(k, 0, p);
        const TcPlanDev& D = many[p];
        if (p != loaded) {   // every warp reaches this point together
            __syncthreads();
            const int prog_ints = 2 * D.n_pairs + D.n_stages + 1;
            for (int i = tid; i < prog_ints; i += blockDim.x) s_prog[i] = D.prog[i];
            for (int i = tid; i < D.n_items * 64; i += blockDim.x) s_gather[i] = D.gather[i];
            __syncthreads();
            loaded = p;
        }
        for (int j = 0; j < kPer; ++j) {
            float* buf = wbuf + cur * 8 * rs;
            const bool has_next = j + 1 < kPer || k + 1 < my_units;
            int pn = 0;
            long long rn = 0;
            if (has_next) rn = step_row0(j + 1 < kPer ? k : k + 1, j + 1 < kPer ? j + 1 : 0, pn);
            if (nbuf == 2 && has_next) pack_issue(many[pn], rn, wbuf + (cur ^ 1) * 8 * rs, rs, lane);
            else asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            __syncwarp();
            int pc;
            const long long row0 = step_row0(k, j, pc);
            const long long tile = row0 / kTcM;
            pack_group(D, buf, rs, row0, tile, (int)(row0 - tile * kTcM), s_prog, s_prog + 2 * D.n_pairs, s_gather,
                       fp16, split, lane);
            if (nbuf == 2) cur ^= 1;
            else if (has_next) pack_issue(many[pn], rn, wbuf, rs, lane);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

struct TcPlan {
    int n = 0, n_leaves = 0, n_groups = 0, n_items = 0, n_stages = 0, gmap_ints = 0;
    unsigned total_b = 0;   // bytes of all hi B images
    TcLeaf* d_leaves = nullptr;
    TcItem* d_items = nullptr;
    int* d_gmap = nullptr;             // output maps per leaf group (see TcArgs::gmap)
    __nv_bfloat16* d_bhi = nullptr;
    __nv_bfloat16* d_blo = nullptr;
    __half* d_fhi = nullptr;
    __half* d_flo = nullptr;
    short* d_gather = nullptr;         // [items][64]: slot feeding each K index (-1: padding)
    TcScratch own;                     // the plan's scratch for its own transforms
    ~TcPlan() {
        for (void* p : {(void*)d_leaves, (void*)d_items, (void*)d_gmap, (void*)d_bhi,
                        (void*)d_blo, (void*)d_fhi,
                        (void*)d_flo, (void*)d_gather})
            if (p) cudaFree(p);
    }
};

template <class T>
T* upload(const std::vector<T>& v) {
    T* d = nullptr;
    GFT_CUDA(cudaMalloc(&d, sizeof(T) * std::max<size_t>(1, v.size())));
    if (!v.empty()) GFT_CUDA(cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return d;
}

uint16_t bf16_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t r = ((u >> 16) & 1u) + 0x7FFFu;  // round to nearest even
    return (uint16_t)((u + r) >> 16);
}
float bf16_val(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

bool tc_eligible(const gft_plan_s& p) {
    if (p.right) return false;   // right Haar units: CUDA-core kernels only
    for (auto& lf : p.leaves)
        if (lf.m() > kTcMaxN) return false;
    return p.n >= 2;
}

// host preparation: leaves, TMEM column groups, coefficient map, stage
// terms, and the pre-split B images (BF16 hi/lo and FP16 hi/lo)
void tc_build(gft_plan_s& p) {
    if (!tc_eligible(p)) return;
    TcPlan* T = new TcPlan;
    try {
        const int n = p.n;
        T->n = n;
        T->n_leaves = (int)p.leaves.size();
        std::vector<TcLeaf> L;
        int off = 0, cols = 0, group = 0;
        long long boff = 0;
        for (auto& lf : p.leaves) {
            TcLeaf t{};
            t.m = lf.m();
            t.npad = std::max(16, (t.m + 15) & ~15);
            t.kchunks = (t.m + kTcK - 1) / kTcK;
            t.off = off;
            if (cols + t.npad > kTcGroupCols) {
                ++group;
                cols = 0;
            }
            t.tcol = cols;
            t.group = group;
            cols += t.npad;
            t.b_off = boff;
            boff += (long long)t.kchunks * t.npad * kTcK;
            off += t.m;
            L.push_back(t);
        }
        T->n_groups = group + 1;
        // output maps: for each leaf group, its coefficients in ascending
        // output position with their TMEM columns; group offsets; first item
        // of each group (items are in leaf order, groups are leaf ranges)
        std::vector<int> gmap;
        {
            std::vector<std::vector<std::pair<int, int>>> per(T->n_groups);
            int i = 0;
            for (size_t k = 0; k < p.leaves.size(); ++k)
                for (int c = 0; c < p.leaves[k].m(); ++c, ++i) per[L[k].group].push_back({p.out_pos[i], L[k].tcol + c});
            std::vector<int> pos, col, goff(1, 0);
            for (auto& v : per) {
                std::sort(v.begin(), v.end());
                for (auto& e : v) {
                    pos.push_back(e.first);
                    col.push_back(e.second);
                }
                goff.push_back((int)pos.size());
            }
            gmap = pos;
            gmap.insert(gmap.end(), col.begin(), col.end());
            gmap.insert(gmap.end(), goff.begin(), goff.end());
        }
        // B images: for each leaf and K chunk, npad rows (outputs c) x 64 K
        // (inputs r) in the smem core-matrix order; B[c][r] = M_k[r][c]
        std::vector<uint16_t> bhi(boff, 0), blo(boff, 0), fhi(boff, 0), flo(boff, 0);
        for (size_t k = 0; k < p.leaves.size(); ++k) {
            const Leaf& lf = p.leaves[k];
            const TcLeaf& t = L[k];
            const int m = lf.m();
            for (int kc = 0; kc < t.kchunks; ++kc)
                for (int c = 0; c < t.npad; ++c)
                    for (int kk = 0; kk < kTcK; ++kk) {
                        const int r = kc * kTcK + kk;
                        double val = 0.0;
                        if (r < m && c < m) val = lf.fold(r, c);
                        const size_t o = (size_t)t.b_off + (size_t)kc * t.npad * kTcK +
                                         (size_t)(((c >> 3) * 8 + (kk >> 3)) * 64 + (c & 7) * 8 + (kk & 7));
                        const float f = (float)val;
                        const uint16_t h = bf16_bits(f);
                        bhi[o] = h;
                        blo[o] = bf16_bits((float)(val - (double)bf16_val(h)));
                        const __half fh = __float2half_rn(f);
                        const __half fl = __float2half_rn((float)(val - (double)__half2float(fh)));
                        fhi[o] = __half_as_ushort(fh);
                        flo[o] = __half_as_ushort(fl);
                    }
        }
        std::vector<TcItem> items;
        unsigned bres = 0;
        for (size_t k = 0; k < L.size(); ++k)
            for (int kc = 0; kc < L[k].kchunks; ++kc) {
                items.push_back({(int)k, kc, (int)bres});
                bres += (unsigned)L[k].npad * kTcK * 2u;
            }
        T->total_b = bres;
        T->n_items = (int)items.size();
        {
            std::vector<short> gat(items.size() * 64, -1);
            for (size_t it = 0; it < items.size(); ++it) {
                const TcLeaf& t = L[items[it].leaf];
                const Leaf& lf = p.leaves[items[it].leaf];
                for (int k = 0; k < 64; ++k) {
                    const int c = items[it].kc * kTcK + k;
                    if (c < t.m) gat[it * 64 + k] = (short)lf.labels[c];
                }
            }
            T->d_gather = upload(gat);
        }
        T->n_stages = p.n_stages;
        T->d_items = upload(items);
        T->d_leaves = upload(L);
        {
            // first item of each group, appended to the output maps
            std::vector<int> gitem(T->n_groups + 1, (int)items.size());
            for (int it = (int)items.size() - 1; it >= 0; --it) gitem[L[items[it].leaf].group] = it;
            for (int g = T->n_groups - 1; g >= 0; --g) gitem[g] = std::min(gitem[g], gitem[g + 1]);
            gmap.insert(gmap.end(), gitem.begin(), gitem.end());
            T->d_gmap = upload(gmap);
            T->gmap_ints = (int)gmap.size();
        }
        T->d_bhi = reinterpret_cast<__nv_bfloat16*>(upload(bhi));
        T->d_blo = reinterpret_cast<__nv_bfloat16*>(upload(blo));
        T->d_fhi = reinterpret_cast<__half*>(upload(fhi));
        T->d_flo = reinterpret_cast<__half*>(upload(flo));
    } catch (...) {
        delete T;
        throw;
    }
    p.tc = T;
}

void tc_free(gft_plan_s& p) {
    delete static_cast<TcPlan*>(p.tc);
    p.tc = nullptr;
}

// Scratch for batches of up to `batch` signals (A images, FP16 scales,
// leaf-ordered output in group mode); grows only.  Reserved before a launch
// that is captured in a CUDA graph, where allocation is not possible.
void tc_reserve(gft_plan_s& p, TcScratch& S, int64_t batch) {
    if (!p.tc && tc_eligible(p)) tc_build(p);
    const TcPlan* T = static_cast<const TcPlan*>(p.tc);
    if (!T || (size_t)batch <= S.rows_cap) return;
    S.release();
    const long long tiles_cap = (batch + kTcM - 1) / kTcM;
    GFT_CUDA(cudaMalloc(&S.d_aimg, (size_t)tiles_cap * T->n_items * 32768u));
    GFT_CUDA(cudaMalloc(&S.d_scale, sizeof(float) * (size_t)batch));
    S.rows_cap = (size_t)batch;
}

void TcScratch::release() {
    for (void** q : {(void**)&d_aimg, (void**)&d_scale, (void**)&d_z})
        if (*q) {
            cudaFree(*q);
            *q = nullptr;
        }
    rows_cap = 0;
}

namespace {

TcPlanDev make_plan_dev(const gft_plan_s& p, const float* x, float* y, int64_t batch, unsigned char* aimg,
                        float* scale, uint32_t precision) {
    const TcPlan* T = static_cast<const TcPlan*>(p.tc);
    TcPlanDev D{};
    D.x = x;
    D.y = y;
    D.aimg = aimg;
    D.scale = scale;
    D.batch = batch;
    D.items = T->d_items;
    D.leaves = T->d_leaves;
    D.gmap = T->d_gmap;
    D.gather = T->d_gather;
    D.prog = p.dev.d_ints;
    const bool f16 = precision == GFT_PREC_FP16X3;
    D.bhi = reinterpret_cast<const unsigned char*>(f16 ? (const void*)T->d_fhi : (const void*)T->d_bhi);
    D.blo = reinterpret_cast<const unsigned char*>(f16 ? (const void*)T->d_flo : (const void*)T->d_blo);
    D.n = p.n;
    D.n_items = T->n_items;
    D.n_leaves = T->n_leaves;
    D.n_groups = T->n_groups;
    D.n_pairs = p.dev.n_pairs;
    D.n_stages = p.dev.n_stages;
    D.total_b = T->total_b;
    return D;
}

int npad_max_of(const gft_plan_s& p) {
    int v = 16;
    for (auto& lf : p.leaves) v = std::max(v, (lf.m() + 15) & ~15);
    return v;
}

void launch_pack(const TcPlanDev& one, const TcPlanDev* many, int n_plans, long long total_tiles, int nmax,
                 int prog_cap, int items_cap, uint32_t precision, cudaStream_t st) {
    if (total_tiles == 0) return;
    // row stride of the staging buffers: a multiple of four floats, so that
    // the 16-byte copies of plans with n % 4 == 0 land 16-byte aligned in
    // every row even when the largest plan of the launch has n % 4 != 0
    const int rs = ((nmax + 3) & ~3) + 4;
    const size_t per_buf = sizeof(float) * (size_t)kPack8Warps * 8 * rs;
    const size_t tabs = sizeof(int) * (size_t)((prog_cap + 3) & ~3) + sizeof(short) * 64 * (size_t)items_cap;
    const int nbuf = 2 * per_buf + tabs <= 232448 / 2 ? 2 : 1;   // double buffer if two CTAs still fit
    const size_t smem = nbuf * per_buf + tabs;
    if (smem > 232448) fail(GFT_ERR_UNSUPPORTED, "tensor-core pack stage does not fit in shared memory");
    if (!many) {
        GFT_CUDA(cudaFuncSetAttribute(tc_pack8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_pack8_kernel, kPack8Warps * 32, smem));
        const long long groups = total_tiles * (kTcM / 8);
        const long long blocks = std::min<long long>((groups + kPack8Warps - 1) / kPack8Warps,
                                                     (long long)std::max(1, per_sm) * sm_count());
        tc_pack8_kernel<<<(unsigned)blocks, kPack8Warps * 32, smem, st>>>(one, rs, nbuf, (int)precision);
    } else {
        GFT_CUDA(cudaFuncSetAttribute(tc_pack8_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_pack8_multi_kernel, kPack8Warps * 32, smem));
        const long long blocks = std::min<long long>(total_tiles, (long long)std::max(1, per_sm) * sm_count());
        tc_pack8_multi_kernel<<<(unsigned)blocks, kPack8Warps * 32, smem, st>>>(many, n_plans, total_tiles, rs, prog_cap,
                                                                              (int)precision, nbuf);
    }
    GFT_CUDA(cudaGetLastError());
}

// resident_b: bytes of all B images of a single plan (0: stream them per item)
void launch_leaf(const TcPlanDev& one, const TcPlanDev* many, int n_plans, long long total_tiles, int npad_max,
                 unsigned resident_b, uint32_t precision, int* err, cudaStream_t st) {
    if (total_tiles == 0) return;
    const bool split = precision != GFT_PREC_BF16;
    const size_t meta = many ? 0
                             : ((sizeof(TcItem) * one.n_items + 15) & ~size_t(15)) +
                                   ((sizeof(TcLeaf) * one.n_leaves + 15) & ~size_t(15)) +
                                   sizeof(int) * (size_t)((2 * one.n + 2 * (one.n_groups + 1) + 3) & ~3);
    const size_t stage = sizeof(float) * (size_t)kTcEpiWarps * 32 * kStageLd + meta;   // staging, then the tables
    const size_t limit = 232448 - 2048;   // leave room for static shared memory
    TcRing ring{};
    const unsigned res_bytes = resident_b * (split ? 2u : 1u);
    if (!many && resident_b && 4u * 32768u + (size_t)res_bytes + stage <= limit) {
        ring.resident = 1;   // all B images once per CTA, four A buffers
        ring.nbuf = 4;
        ring.bufsz = 32768u;
        ring.res_off = 4u * 32768u;
        ring.stage_off = (unsigned)((ring.res_off + res_bytes + 15) & ~size_t(15));
    } else {
        ring.resident = 0;   // A and the item's B images in each buffer
        ring.bslot = 32768u;
        const unsigned bb = (unsigned)npad_max * kTcK * 2u * (split ? 2u : 1u);
        ring.bufsz = (32768u + bb + 1023u) & ~1023u;
        ring.nbuf = (int)std::min<size_t>(4, (limit - stage) / ring.bufsz);
        if (ring.nbuf < 2) fail(GFT_ERR_UNSUPPORTED, "tensor-core kernel does not fit in shared memory");
        ring.res_off = 0;
        ring.stage_off = (unsigned)ring.nbuf * ring.bufsz;
    }
    ring.meta_off = ring.stage_off + (unsigned)(sizeof(float) * (size_t)kTcEpiWarps * 32 * kStageLd);
    const size_t smem = ring.stage_off + stage;
    if (smem > limit) fail(GFT_ERR_UNSUPPORTED, "tensor-core kernel does not fit in shared memory");
    GFT_CUDA(cudaFuncSetAttribute(tc_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<long long>(total_tiles, sm_count());
    tc_leaf_kernel<<<grid, kTcThreads, smem, st>>>(one, many, n_plans, total_tiles, (int)precision, err, ring);
    GFT_CUDA(cudaGetLastError());
}

}  // namespace

void launch_tc(gft_plan_s& p, const float* x, float* y, int64_t batch, bool inverse, cudaStream_t st,
               uint32_t precision, TcScratch* scratch) {
    if (inverse) fail(GFT_ERR_UNSUPPORTED, "tensor-core precisions are implemented for the forward transform");
    if (!p.tc && tc_eligible(p)) tc_build(p);   // built on first use
    if (!p.tc && p.right) fail(GFT_ERR_UNSUPPORTED, "tensor-core precisions do not run bipartite plans (right Haar units)");
    if (!p.tc) fail(GFT_ERR_UNSUPPORTED, "tensor-core path needs every leaf to have at most 256 nodes");
    if (x == y) fail(GFT_ERR_UNSUPPORTED, "tensor-core path does not run in place");
    TcPlan* T = static_cast<TcPlan*>(p.tc);
    TcScratch& S = scratch ? *scratch : T->own;
    tc_reserve(p, S, batch);
    const long long n_tiles = (batch + kTcM - 1) / kTcM;
    const TcPlanDev D = make_plan_dev(p, x, y, batch, S.d_aimg, S.d_scale, precision);
    launch_pack(D, nullptr, 1, n_tiles, p.n, 2 * p.dev.n_pairs + p.dev.n_stages + 1, T->n_items, precision, st);
    launch_leaf(D, nullptr, 1, n_tiles, npad_max_of(p), T->total_b, precision, p.dev.d_err, st);
}

// ---------------------------------------------------------------------------
// mixed batches: all tensor-core plans of a batch in one pack launch and one
// leaf launch per size class (n <= 256, n > 256: the pack stage's shared
// staging is sized by the class's largest graph)
// ---------------------------------------------------------------------------
namespace {
struct TcBatch {
    uint32_t prec = 0;
    struct Class {
        std::vector<TcPlanDev> desc;
        std::vector<int> user;           // index in the caller's list
        TcPlanDev* d_desc = nullptr;
        long long total_tiles = 0, total_groups = 0;
        int nmax = 0, npad_max = 16, prog_cap = 1, items_cap = 1;
        int* err = nullptr;
    } cls[2];
    unsigned char* d_aimg = nullptr;
    float* d_scale = nullptr;
    ~TcBatch() {
        for (auto& c : cls)
            if (c.d_desc) cudaFree(c.d_desc);
        if (d_aimg) cudaFree(d_aimg);
        if (d_scale) cudaFree(d_scale);
    }
};
}  // namespace

void* tc_batch_create(const std::vector<gft_plan_s*>& plans, const std::vector<int64_t>& batches,
                      uint32_t precision) {
    std::unique_ptr<TcBatch> B(new TcBatch);
    B->prec = precision;
    size_t aimg_bytes = 0, scale_elems = 0;
    std::vector<size_t> a_off(plans.size()), s_off(plans.size());
    for (size_t i = 0; i < plans.size(); ++i) {
        gft_plan_s& p = *plans[i];
        if (!p.tc && tc_eligible(p)) tc_build(p);
        if (!p.tc) fail(GFT_ERR_UNSUPPORTED, "tensor-core path needs every leaf to have at most 256 nodes");
        const TcPlan* T = static_cast<const TcPlan*>(p.tc);
        const long long tiles = (batches[i] + kTcM - 1) / kTcM;
        a_off[i] = aimg_bytes;
        s_off[i] = scale_elems;
        aimg_bytes += (size_t)tiles * T->n_items * 32768u;
        scale_elems += (size_t)batches[i];
    }
    GFT_CUDA(cudaMalloc(&B->d_aimg, std::max<size_t>(aimg_bytes, 256)));
    GFT_CUDA(cudaMalloc(&B->d_scale, sizeof(float) * std::max<size_t>(scale_elems, 1)));
    for (size_t i = 0; i < plans.size(); ++i) {
        gft_plan_s& p = *plans[i];
        TcBatch::Class& c = B->cls[p.n > 256 ? 1 : 0];
        TcPlanDev D = make_plan_dev(p, nullptr, nullptr, batches[i], B->d_aimg + a_off[i], B->d_scale + s_off[i],
                                    precision);
        const long long tiles = (batches[i] + kTcM - 1) / kTcM;
        D.tile0 = c.total_tiles;
        D.group0 = c.total_groups;
        c.total_tiles += tiles;
        c.total_groups += tiles * (kTcM / 8);
        c.nmax = std::max(c.nmax, p.n);
        c.npad_max = std::max(c.npad_max, npad_max_of(p));
        c.prog_cap = std::max(c.prog_cap, 2 * p.dev.n_pairs + p.dev.n_stages + 1);
        c.items_cap = std::max(c.items_cap, D.n_items);
        if (!c.err) c.err = p.dev.d_err;
        c.desc.push_back(D);
        c.user.push_back((int)i);
    }
    for (auto& c : B->cls)
        if (!c.desc.empty()) GFT_CUDA(cudaMalloc(&c.d_desc, sizeof(TcPlanDev) * c.desc.size()));
    return B.release();
}

void tc_batch_upload(void* h, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st) {
    TcBatch* B = static_cast<TcBatch*>(h);
    for (auto& c : B->cls) {
        if (c.desc.empty()) continue;
        for (size_t j = 0; j < c.desc.size(); ++j) {
            c.desc[j].x = x[c.user[j]];
            c.desc[j].y = y[c.user[j]];
        }
        GFT_CUDA(cudaMemcpyAsync(c.d_desc, c.desc.data(), sizeof(TcPlanDev) * c.desc.size(), cudaMemcpyHostToDevice, st));
    }
}

void tc_batch_launch(void* h, cudaStream_t st) {
    TcBatch* B = static_cast<TcBatch*>(h);
    for (auto& c : B->cls) {
        if (c.desc.empty()) continue;
        const TcPlanDev none{};
        launch_pack(none, c.d_desc, (int)c.desc.size(), c.total_tiles, c.nmax, c.prog_cap, c.items_cap, B->prec, st);
        launch_leaf(none, c.d_desc, (int)c.desc.size(), c.total_tiles, c.npad_max, 0, B->prec, c.err, st);
    }
}

void tc_batch_free(void* h) { delete static_cast<TcBatch*>(h); }

int tc_batch_launches(void* h) {
    int n = 0;
    for (auto& c : static_cast<TcBatch*>(h)->cls)
        if (!c.desc.empty() && c.total_tiles > 0) n += 2;   // pack + leaf
    return n;
}

}  // namespace gft

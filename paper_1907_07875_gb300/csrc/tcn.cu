// Tensor-core leaf products for batches of many graphs with FEW signals
// each (the size sweep: 10^4 graphs of 8..1024 nodes, a few dozen to a few
// hundred signals per graph), leaves up to 512 nodes.
//
// The leaf products y_k = M_k^T v_k (Sec. IV-C, Eq. 13; M_k the folded leaf
// basis) of a tile of NS signals run with the roles of the operands swapped
// against tc.cu: the MMA's M axis is the leaf's output coefficients (128 per
// M-tile), its N axis the tile's signals (NS = 16 or 32), K the leaf's
// inputs:
//     D[c][s] (TMEM lane c, column s) = sum_r M_k[r][c] v_k[r][s]
// so a graph with 27 signals fills a 32-column accumulator instead of 27 of
// 128 rows, and a 512-node leaf is four M-tiles sharing one B operand.
//
// Per CTA (persistent, tiles b, b + grid, ...), warp-specialised:
//   warps 0-3 (workers): copy the tile's NS signal rows into shared memory
//     (cp.async), compute the FP16 per-signal scales, run the Haar stages in
//     place (FP32), and write the B operand of EVERY (leaf, 32-wide K chunk)
//     of the tile -- the gathered post-stage values, split into hi and lo
//     (BF16 or scaled FP16), in the canonical no-swizzle K-major layout --
//     into a resident region; then signal the MMA thread.  After the tile's
//     last MMA they read the accumulators (tcgen05.ld, warp w = TMEM lanes
//     32w..32w+31), scatter them to their output positions (ascending
//     eigenvalue) in a staging copy of the tile's output rows, and write the
//     rows with coalesced 16-byte stores;
//   warp 4 (one thread): streams the pre-split basis chunks A = M_k^T
//     (128 rows x 32 K, hi and lo, 8 KB each) through a ring of shared-memory
//     slots with bulk copies (TMA), running ahead across tiles;
//   warp 5: allocates TMEM (256 columns); one thread issues the MMAs
//     (M = 128, N = NS, K = 16; hi*hi + hi*lo + lo*hi for the split
//     precisions) into one NS-column accumulator per (leaf, M-tile), and
//     commits each ring slot back to the copier and the tile's accumulators
//     to the workers.
// Every wait is bounded (about 2 s via %globaltimer); a timeout records
// GFT_ERR_TIMEOUT in the error word, every role leaves its loop through
// uniform exits (workers agree through a barrier reduction), copies and MMAs
// in flight are awaited (bounded), and TMEM is freed.
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
constexpr int kNK = 32;              // K per basis chunk
constexpr int kNWorkers = 4;         // worker warps 0-3
constexpr int kNThreads = 192;       // + copier warp 4, MMA warp 5
constexpr int kNSlots = 3;           // ring slots (A hi + A lo, 8 KB each)
constexpr int kNCols = 256;          // TMEM columns per CTA (two CTAs per SM fit)
constexpr int kNMaxLeaf = 512;
constexpr unsigned kNSlotBytes = 2u * kNM * kNK * 2u;   // 16 KB
constexpr unsigned long long kNWaitNs = 2000000000ull;

struct TcnLeaf {
    int m;          // leaf size
    int npad;       // rows of the basis image (m rounded up to 16)
    int kchunks;    // ceil(m / 32)
    int mtiles;     // ceil(npad / 128)
    int lab;        // offset of the leaf's nodes in the plan's leaf-ordered label / output-position lists
    int kc0;        // first B chunk of this leaf within a tile
    int unit0;      // first accumulator (M-tile) of this leaf within a tile
    int pad;
    long long a_off;   // element offset of the leaf's basis images
};

struct TcnPlanDev {
    const float* x;
    float* y;
    long long batch;
    long long tile0;           // first tile of this plan in the launch
    const int* prog;           // [pairs 2P][stage offsets S+1][labels n][out_pos n] ...
    const TcnLeaf* leaves;
    const unsigned char* ahi;  // basis images of this launch's precision
    const unsigned char* alo;
    int* err;                  // the plan's device error word
    int n, np, ns, n_leaves, n_units, n_chunks, n_stages, n_pairs;
    int off_labels, off_outpos;
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
// barrier 1 over the four worker warps with an OR reduction: every worker
// gets the same answer, so exits taken on it are uniform
__device__ __forceinline__ bool workers_any(bool v) {
    unsigned r;
    asm volatile("{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.or.pred q, 1, 128, p; selp.u32 %0, 1, 0, q; }"
                 : "=r"(r)
                 : "r"((unsigned)v)
                 : "memory");
    return r != 0;
}
__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// byte offset of (row, K group) in a [rows x 32] K-major no-swizzle image
// whose 8-row groups are 512 B apart (4 K groups of 16 B per row)
__device__ __forceinline__ unsigned coff(int row, int kg) {
    return (unsigned)(((row >> 3) * 4 + kg) * 128 + (row & 7) * 16);
}

template <bool TILES>
__device__ __forceinline__ int plan_of_tile(const TcnPlanDev* P, int n_plans, long long t) {
    int lo = 0, hi = n_plans - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace
}  // namespace gft

namespace gft {
namespace {

// Persistent kernel over the tiles of every plan of one launch (plan order;
// CTA b takes tiles b, b + grid, ...).  Dynamic shared memory:
//   [ring: kNSlots x (A hi 8 KB | A lo 8 KB)]
//   [B region: per (leaf, K chunk) of a tile, hi (ns x 64 B) then lo]
//   [tile: ns rows x np floats -- input, then output staging][scales: 32 floats]
__global__ void __launch_bounds__(kNThreads, 1) tcn_kernel(const TcnPlanDev* __restrict__ plans, int n_plans,
                                                          long long total_tiles, int prec, unsigned b_bytes,
                                                          unsigned tile_floats) {
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* ring = sm;
    unsigned char* breg = sm + kNSlots * kNSlotBytes;
    float* tile = reinterpret_cast<float*>(breg + b_bytes);
    float* s_scale = tile + tile_floats;
    __shared__ __align__(8) unsigned long long a_full[kNSlots], empty[kNSlots], b_ready, acc_full, drain;
    __shared__ unsigned s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"(kNCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kNSlots; ++i) {
            bar_init(&a_full[i], 1);
            bar_init(&empty[i], 1);
        }
        bar_init(&b_ready, kNWorkers);
        bar_init(&acc_full, 1);
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
    const long long my_tiles = total_tiles > blockIdx.x ? (total_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto abort_now = [&](int* err) {
        s_abort = 1;
        atomicExch(err, (int)GFT_ERR_TIMEOUT);
    };

    if (warp == kNWorkers) {
        // ---------------- basis chunks (TMA) ----------------
        if (lane == 0) {
            long long q = 0;
            bool issued[kNSlots] = {};
            unsigned par[kNSlots] = {};
            bool stop = false;
            for (long long j = 0; j < my_tiles && !stop; ++j) {
                const long long t = blockIdx.x + j * (long long)gridDim.x;
                const TcnPlanDev& D = plans[plan_of_tile<true>(plans, n_plans, t)];
                for (int k = 0; k < D.n_leaves && !stop; ++k) {
                    const TcnLeaf L = D.leaves[k];
                    for (int mt = 0; mt < L.mtiles && !stop; ++mt) {
                        const unsigned bytes = (unsigned)min(kNM, L.npad - mt * kNM) * kNK * 2u;
                        for (int kc = 0; kc < L.kchunks; ++kc, ++q) {
                            const int s = (int)(q % kNSlots);
                            const long long use = q / kNSlots;
                            if (s_abort || (use >= 1 && !bar_wait(&empty[s], (unsigned)((use - 1) & 1)))) {
                                abort_now(D.err);
                                stop = true;
                                break;
                            }
                            unsigned char* dst = ring + (size_t)s * kNSlotBytes;
                            const size_t src =
                                2 * (size_t)(L.a_off + (long long)kc * L.npad * kNK + (long long)mt * kNM * kNK);
                            bar_expect(&a_full[s], split ? 2 * bytes : bytes);
                            bulk(dst, D.ahi + src, bytes, &a_full[s]);
                            if (split) bulk(dst + kNSlotBytes / 2, D.alo + src, bytes, &a_full[s]);
                            issued[s] = true;
                            par[s] = (unsigned)(use & 1);
                        }
                    }
                }
            }
            for (int s = 0; s < kNSlots; ++s)   // no copy left in flight
                if (issued[s]) bar_wait(&a_full[s], par[s]);
        }
    } else if (warp == kNWorkers + 1) {
        // ---------------- MMAs ----------------
        if (lane == 0) {
            long long q = 0;
            bool stop = false;
            for (long long j = 0; j < my_tiles && !stop; ++j) {
                const long long t = blockIdx.x + j * (long long)gridDim.x;
                const TcnPlanDev& D = plans[plan_of_tile<true>(plans, n_plans, t)];
                if (s_abort || !bar_wait(&b_ready, (unsigned)(j & 1))) {
                    abort_now(D.err);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int ns = D.ns;
                const unsigned id = idesc(ns, !fp16);
                const unsigned bbase = su32(breg);
                for (int k = 0; k < D.n_leaves && !stop; ++k) {
                    const TcnLeaf L = D.leaves[k];
                    const int kmax = (L.m + 15) & ~15;
                    for (int mt = 0; mt < L.mtiles && !stop; ++mt) {
                        const unsigned dt = tmem + (unsigned)((L.unit0 + mt) * ns);
                        for (int kc = 0; kc < L.kchunks; ++kc, ++q) {
                            const int s = (int)(q % kNSlots);
                            if (s_abort || !bar_wait(&a_full[s], (unsigned)((q / kNSlots) & 1))) {
                                abort_now(D.err);
                                stop = true;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const unsigned abase = su32(ring + (size_t)s * kNSlotBytes);
                            const unsigned bch = bbase + (unsigned)((L.kc0 + kc) * ns * 128);
                            for (int ks = 0; ks < kNK / 16; ++ks) {
                                if (kc * kNK + ks * 16 >= kmax) break;
                                const unsigned koff = ks * 256u;
                                const unsigned long long ah = sdesc(abase + koff, 128, 512);
                                const unsigned long long bh = sdesc(bch + koff, 128, 512);
                                mma(dt, ah, bh, id, (kc | ks) ? 1u : 0u);
                                if (split) {
                                    mma(dt, ah, sdesc(bch + (unsigned)(ns * 64) + koff, 128, 512), id, 1u);
                                    mma(dt, sdesc(abase + kNSlotBytes / 2 + koff, 128, 512), bh, id, 1u);
                                }
                            }
                            commit_to(&empty[s]);
                        }
                    }
                }
                if (!stop) commit_to(&acc_full);
            }
            commit_to(&drain);             // arrives once every MMA issued above is complete
            bar_wait(&drain, 0);
        }
    } else {
        // ---------------- workers (warps 0-3) ----------------
        const int wt = tid;
        for (long long j = 0; j < my_tiles; ++j) {
            const long long t = blockIdx.x + j * (long long)gridDim.x;
            const TcnPlanDev D = plans[plan_of_tile<true>(plans, n_plans, t)];
            const int n = D.n, np = D.np, ns = D.ns;
            const long long tp = t - D.tile0;
            const int rows = (int)min((long long)ns, D.batch - tp * ns);
            const int* labels = D.prog + D.off_labels;
            const int* outpos = D.prog + D.off_outpos;
            // 1. signal rows -> tile (row stride np)
            const float* src = D.x + tp * ns * (long long)n;
            if ((n & 3) == 0) {
                const int per = n >> 2;
                for (int e = wt; e < rows * per; e += 128) {
                    const int s = e / per, c4 = e - s * per;
                    const unsigned d = su32(tile + s * np + 4 * c4);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + (long long)s * n + 4 * c4)
                                 : "memory");
                }
            } else {
                for (int e = wt; e < rows * n; e += 128) {
                    const int s = e / n, c = e - s * n;
                    const unsigned d = su32(tile + s * np + c);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src + e) : "memory");
                }
            }
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
            workers_sync();
            // 2. per-signal scales (FP16: a power of two bounding the post-stage values)
            for (int s = warp; s < 32; s += kNWorkers) {
                float mx = 0.f;
                if (fp16 && s < rows)
                    for (int c = lane; c < n; c += 32) mx = fmaxf(mx, fabsf(tile[s * np + c]));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if (lane == 0) s_scale[s] = mx > 0.f ? exp2f(ceilf(log2f(mx)) + (float)D.n_stages) : 1.f;
            }
            // 3. Haar stages in place (Sec. III; the 1/sqrt2 factors are in the basis)
            for (int st = 0; st < D.n_stages; ++st) {
                const int p0 = D.prog[2 * D.n_pairs + st], cnt = D.prog[2 * D.n_pairs + st + 1] - p0;
                for (int e = wt; e < rows * cnt; e += 128) {
                    const int s = e / cnt, pp = p0 + (e - s * cnt);
                    const int i = D.prog[2 * pp], jj = D.prog[2 * pp + 1];
                    float* row = tile + s * np;
                    const float u = row[i], v = row[jj];
                    row[i] = u + v;
                    row[jj] = u - v;
                }
                workers_sync();
            }
            workers_sync();   // scales visible
            // 4. B operand of every (leaf, K chunk): rows = signals, hi then lo
            const int groups = ns >> 3;
            for (int k = 0; k < D.n_leaves; ++k) {
                const TcnLeaf L = D.leaves[k];
                const int total = L.kchunks * groups * 32;
                for (int e = wt; e < total; e += 128) {
                    const int slo = e & 7, kg = (e >> 3) & 3, rest = e >> 5;
                    const int rg = rest % groups, kc = rest / groups;
                    const int s = rg * 8 + slo;
                    const bool live = s < rows;
                    const float inv = fp16 ? 1.f / s_scale[s] : 1.f;
                    const int r0 = kc * kNK + kg * 8;
                    float v[8];
#pragma unroll
                    for (int ee = 0; ee < 8; ++ee) {
                        const int r = r0 + ee;
                        v[ee] = (live && r < L.m) ? tile[s * np + labels[L.lab + r]] * inv : 0.f;
                    }
                    unsigned hi[4], lo[4];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        if (fp16) {
                            const __half2 h = __floats2half2_rn(v[2 * qq], v[2 * qq + 1]);
                            const float2 hf = __half22float2(h);
                            const __half2 l = __floats2half2_rn(v[2 * qq] - hf.x, v[2 * qq + 1] - hf.y);
                            hi[qq] = *reinterpret_cast<const unsigned*>(&h);
                            lo[qq] = *reinterpret_cast<const unsigned*>(&l);
                        } else {
                            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * qq], v[2 * qq + 1]);
                            const float2 hf = __bfloat1622float2(h);
                            const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * qq] - hf.x, v[2 * qq + 1] - hf.y);
                            hi[qq] = *reinterpret_cast<const unsigned*>(&h);
                            lo[qq] = *reinterpret_cast<const unsigned*>(&l);
                        }
                    }
                    unsigned char* dst = breg + (size_t)(L.kc0 + kc) * ns * 128 + coff(s, kg);
                    *reinterpret_cast<uint4*>(dst) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    if (split) *reinterpret_cast<uint4*>(dst + ns * 64) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
            // generic-proxy writes of the B region -> visible to the tensor cores
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            workers_sync();
            if (lane == 0) bar_arrive(&b_ready);
            // 5. wait for the tile's accumulators (uniform exit on timeout)
            const bool bad = !bar_wait(&acc_full, (unsigned)(j & 1));
            if (workers_any(bad || s_abort != 0)) {
                if (wt == 0) abort_now(D.err);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // 6. accumulators -> output staging (the tile buffer is free: every
            //    B chunk was built before the MMAs could complete)
            const unsigned lane_base = (unsigned)(warp * 32) << 16;
            for (int k = 0; k < D.n_leaves; ++k) {
                const TcnLeaf L = D.leaves[k];
                for (int mt = 0; mt < L.mtiles; ++mt) {
                    const int c = mt * kNM + warp * 32 + lane;
                    const bool valid = c < L.m;
                    const int pos = valid ? outpos[L.lab + c] : 0;
                    for (int c0 = 0; c0 < ns; c0 += 16) {
                        unsigned r[16];
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                            "[%16];"
                            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                              "=r"(r[14]), "=r"(r[15])
                            : "r"(tmem + lane_base + (unsigned)((L.unit0 + mt) * ns + c0)));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (valid) {
#pragma unroll
                            for (int qq = 0; qq < 16; ++qq) {
                                const int s = c0 + qq;
                                if (s < rows) tile[s * np + pos] = __uint_as_float(r[qq]) * s_scale[s];
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            workers_sync();
            // 7. output rows, coalesced
            float* dst = D.y + tp * ns * (long long)n;
            if ((n & 3) == 0) {
                const int per = n >> 2;
                for (int e = wt; e < rows * per; e += 128) {
                    const int s = e / per, c4 = e - s * per;
                    const float4 v = *reinterpret_cast<const float4*>(tile + s * np + 4 * c4);
                    __stcs(reinterpret_cast<float4*>(dst + (long long)s * n + 4 * c4), v);
                }
            } else {
                for (int e = wt; e < rows * n; e += 128) {
                    const int s = e / n, c = e - s * n;
                    __stcs(dst + e, tile[s * np + c]);
                }
            }
            workers_sync();   // tile buffer free for the next load
        }
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
constexpr size_t kNTwoPerSm = 112 * 1024;   // dynamic + static shared memory for two CTAs per SM
constexpr size_t kNFixed = (size_t)kNSlots * kNSlotBytes + 32 * sizeof(float);

struct TcnPlan {
    std::vector<TcnLeaf> leaves;
    TcnLeaf* d_leaves = nullptr;
    int n_units = 0, n_chunks = 0;
    long long img_elems = 0;
    unsigned char* d_img[2][2] = {};   // [BF16, FP16][hi, lo]
    ~TcnPlan() {
        if (d_leaves) cudaFree(d_leaves);
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

int units_of(const gft_plan_s& p) {
    int u = 0;
    for (auto& lf : p.leaves) u += (((lf.m() + 15) & ~15) + kNM - 1) / kNM;
    return u;
}

TcnPlan* tcn_prepare(gft_plan_s& p) {
    if (p.tcn) return static_cast<TcnPlan*>(p.tcn);
    std::unique_ptr<TcnPlan> T(new TcnPlan);
    int lab = 0, kc0 = 0, unit0 = 0;
    long long a = 0;
    for (auto& lf : p.leaves) {
        TcnLeaf L{};
        L.m = lf.m();
        L.npad = (L.m + 15) & ~15;
        L.kchunks = (L.m + kNK - 1) / kNK;
        L.mtiles = (L.npad + kNM - 1) / kNM;
        L.lab = lab;
        L.kc0 = kc0;
        L.unit0 = unit0;
        L.a_off = a;
        lab += L.m;
        kc0 += L.kchunks;
        unit0 += L.mtiles;
        a += (long long)L.kchunks * L.npad * kNK;
        T->leaves.push_back(L);
    }
    T->n_units = unit0;
    T->n_chunks = kc0;
    T->img_elems = a;
    GFT_CUDA(cudaMalloc(&T->d_leaves, sizeof(TcnLeaf) * T->leaves.size()));
    GFT_CUDA(cudaMemcpy(T->d_leaves, T->leaves.data(), sizeof(TcnLeaf) * T->leaves.size(), cudaMemcpyHostToDevice));
    p.tcn = T.release();
    return static_cast<TcnPlan*>(p.tcn);
}

// basis images of one precision: per leaf and 32-wide K chunk, npad rows
// (output coefficients c) x 32 K (inputs r) in the K-major core-matrix
// order of the kernel; A[c][r] = M_k[r][c], split into hi and lo
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

// signals per tile: 32 when the accumulators fit in TMEM and the tile stays
// small, else 16
int ns_of(const gft_plan_s& p, int64_t batch, int units) {
    if (batch > 16 && units * 32 <= kNCols && (size_t)32 * np_of(p.n) * sizeof(float) <= 32 * 1024) return 32;
    return 16;
}

struct TcnClass {
    std::vector<int> members;            // slot -> index in the batch's plan list
    std::vector<TcnPlanDev> desc;
    TcnPlanDev* d_desc = nullptr;
    long long total_tiles = 0;
    unsigned b_cap = 0, tile_cap = 0;
    size_t smem = 0;
    int grid = 0;
};

struct TcnBatch {
    uint32_t prec = GFT_PREC_BF16X3;
    std::vector<TcnClass> classes;
    ~TcnBatch() {
        for (auto& c : classes)
            if (c.d_desc) cudaFree(c.d_desc);
    }
};

}  // namespace

bool tcn_eligible(const gft_plan_s& p) {
    if (p.right || !p.has_device || p.n < 2) return false;
    for (auto& lf : p.leaves)
        if (lf.m() > kNMaxLeaf) return false;
    if (units_of(p) * 16 > kNCols) return false;
    const size_t bytes = (size_t)16 * 128 * [&] {
        int c = 0;
        for (auto& lf : p.leaves) c += (lf.m() + kNK - 1) / kNK;
        return c;
    }() + (size_t)16 * np_of(p.n) * sizeof(float);
    return kNFixed + bytes + 1024 <= kNSmemLimit;
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
    std::vector<int> cls(k);
    std::vector<double> cost(k);
    for (int i = 0; i < k; ++i) {
        gft_plan_s& p = *plans[i];
        if (!tcn_eligible(p)) fail(GFT_ERR_UNSUPPORTED, "plan not supported by the few-signals tensor-core kernel");
        TcnPlan* T = tcn_prepare(p);
        tcn_images(p, *T, fp16);
        TcnPlanDev& e = d[i];
        e = TcnPlanDev{};
        e.batch = batches[i];
        e.prog = p.dev.d_ints;
        e.leaves = T->d_leaves;
        e.ahi = T->d_img[fp16 ? 1 : 0][0];
        e.alo = T->d_img[fp16 ? 1 : 0][1];
        e.err = p.dev.d_err;
        e.n = p.n;
        e.np = np_of(p.n);
        e.ns = ns_of(p, batches[i], T->n_units);
        e.n_leaves = (int)T->leaves.size();
        e.n_units = T->n_units;
        e.n_chunks = T->n_chunks;
        e.n_stages = p.dev.n_pre_stages;
        e.n_pairs = p.dev.n_pairs;
        e.off_labels = 2 * p.dev.n_pairs + p.dev.n_stages + 1;
        e.off_outpos = e.off_labels + p.n;
        const size_t bytes = (size_t)e.n_chunks * e.ns * 128 + (size_t)e.ns * e.np * sizeof(float);
        cls[i] = kNFixed + bytes + 1024 <= kNTwoPerSm ? 0 : 1;
        double a_chunks = 0;
        for (auto& L : T->leaves) a_chunks += (double)L.mtiles * L.kchunks;
        cost[i] = a_chunks * 16384.0 + (double)e.ns * p.n * 8.0;   // bytes moved per tile
    }
    for (int c = 0; c < 2; ++c) {
        TcnClass C;
        for (int i = 0; i < k; ++i)
            if (cls[i] == c) C.members.push_back(i);
        if (C.members.empty()) continue;
        std::stable_sort(C.members.begin(), C.members.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        for (int i : C.members) {
            TcnPlanDev e = d[i];
            e.tile0 = C.total_tiles;
            C.total_tiles += (e.batch + e.ns - 1) / e.ns;
            C.b_cap = std::max(C.b_cap, (unsigned)(e.n_chunks * e.ns * 128));
            C.tile_cap = std::max(C.tile_cap, (unsigned)(e.ns * e.np));
            C.desc.push_back(e);
        }
        C.tile_cap = (C.tile_cap + 31) & ~31u;
        C.smem = kNFixed + C.b_cap + sizeof(float) * (size_t)C.tile_cap;
        if (C.smem > kNSmemLimit) fail(GFT_ERR_UNSUPPORTED, "few-signals tensor-core batch needs too much shared memory");
        cudaFuncAttributes fa{};
        GFT_CUDA(cudaFuncGetAttributes(&fa, tcn_kernel));
        if (C.smem + fa.sharedSizeBytes > kNSmemLimit)
            fail(GFT_ERR_UNSUPPORTED, "few-signals tensor-core batch needs too much shared memory");
        GFT_CUDA(cudaFuncSetAttribute(tcn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kNSmemLimit - fa.sharedSizeBytes)));
        int per_sm = 0;
        GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tcn_kernel, kNThreads, C.smem));
        if (per_sm < 1) fail(GFT_ERR_UNSUPPORTED, "few-signals tensor-core kernel does not fit on an SM");
        per_sm = std::min(per_sm, 2);   // TMEM: 256 columns per CTA
        C.grid = (int)std::max<long long>(1, std::min<long long>(C.total_tiles, (long long)per_sm * sm_count()));
        B->classes.push_back(std::move(C));   // owned by the batch before the allocation
        TcnClass& D = B->classes.back();
        GFT_CUDA(cudaMalloc(&D.d_desc, sizeof(TcnPlanDev) * D.desc.size()));
    }
    return B.release();
}

void tcn_batch_upload(void* h, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st) {
    TcnBatch* B = static_cast<TcnBatch*>(h);
    for (auto& C : B->classes) {
        for (size_t sl = 0; sl < C.desc.size(); ++sl) {
            C.desc[sl].x = x[C.members[sl]];
            C.desc[sl].y = y[C.members[sl]];
        }
        GFT_CUDA(cudaMemcpyAsync(C.d_desc, C.desc.data(), sizeof(TcnPlanDev) * C.desc.size(), cudaMemcpyHostToDevice, st));
    }
}

void tcn_batch_launch(void* h, cudaStream_t st) {
    TcnBatch* B = static_cast<TcnBatch*>(h);
    for (auto& C : B->classes) {
        if (C.total_tiles == 0) continue;
        tcn_kernel<<<C.grid, kNThreads, C.smem, st>>>(C.d_desc, (int)C.desc.size(), C.total_tiles, (int)B->prec,
                                                       C.b_cap, C.tile_cap);
        GFT_CUDA(cudaGetLastError());
    }
}

void tcn_batch_free(void* h) { delete static_cast<TcnBatch*>(h); }

int tcn_batch_launches(void* h) {
    int n = 0;
    for (auto& c : static_cast<TcnBatch*>(h)->classes) n += c.total_tiles > 0 ? 1 : 0;
    return n;
}

}  // namespace gft

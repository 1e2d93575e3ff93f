// Plan-specialised transform kernels, generated at plan creation and
// compiled with NVRTC for sm_103a.
//
// The interpreter kernel (apply.cu) reads stage pairs, node lists and leaf
// matrices from shared memory and spends most of its instructions on index
// loads and address arithmetic.  For small graphs (n <= 128) the whole plan
// fits in straight-line code, so this generator writes one kernel per plan
// in which every index is a compile-time constant and every leaf-matrix
// entry is an FMA immediate:
//   * each thread loads its signal's n values from the shared tile into
//     registers (vector loads when the row stride allows),
//   * applies the Haar units as register additions / subtractions,
//   * computes each coefficient as an FMA chain over its leaf's inputs
//     (entries that are exactly zero are skipped), and writes the
//     coefficients back over the row in output order, so the store is a
//     plain coalesced copy.
// The tile pipeline (persistent CTAs, cp.async double or single buffering,
// 16-byte streaming stores) is the same as the interpreter's.  Several
// launch shapes are compiled into one module and timed at plan creation;
// the fastest per direction is kept (the autotuner).
#include <nvrtc.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "gft_internal.h"

namespace gft {

namespace {

constexpr int kSmemLimitJ = 232448;
// Plans that get straight-line kernels: a signal's n values live in
// registers (n <= 128 keeps them there under a 255-register cap), and the
// leaf matrices become sum(m^2) FMA immediates per direction (bounds the
// code size and the NVRTC compile time: about 10 s at 8192).  FP64 values
// take two registers and FP64 FMAs are slow on this part, so the FP64
// module is built only for the smaller plans.
constexpr int kJitMaxN = 128;
constexpr int kTuneReps = 5;   // timed launches per candidate shape (after one warm-up)
constexpr long long kJitMaxLeafEntries = 8192;
constexpr long long kJitMaxLeafEntries64 = 4096;

long long leaf_entries(const gft_plan_s& p) {
    long long fl = 0;
    for (auto& lf : p.leaves) fl += (long long)lf.m() * lf.m();
    return fl;
}

struct Cand {
    int rs, threads, nbuf, bulk;
};

// Launch shapes compiled and timed for FP32 (FP64 uses the first only).
// bulk = 1: whole tiles move with cp.async.bulk (TMA) and an mbarrier;
// only for plans whose shared row stride equals n.
const Cand kCands[] = {{2, 64, 1, 0}, {2, 128, 1, 0}, {1, 128, 1, 0}, {2, 128, 2, 0},
                       {1, 128, 1, 1}, {1, 128, 2, 1}, {2, 128, 2, 1}, {2, 64, 2, 1}};

enum RowMode { kContig = 0, kVec4 = 1, kPad1 = 2 };

std::string lit(double v, bool f64) {
    char b[64];
    if (f64) std::snprintf(b, sizeof b, "%a", v);
    else std::snprintf(b, sizeof b, "%af", (double)(float)v);
    return b;
}

const char* kHelpers = R"(
typedef long long i64;
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    unsigned a;
    asm("{ .reg .u64 t; cvta.to.shared.u64 t, %1; cvt.u32.u64 %0, t; }" : "=r"(a) : "l"(p));
    return a;
}
__device__ __forceinline__ void cpa16(void* s, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cpa8(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cpa4(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void stcs(float* p, float v) { asm volatile("st.global.cs.f32 [%0], %1;" :: "l"(p), "f"(v) : "memory"); }
__device__ __forceinline__ void stcs(double* p, double v) { asm volatile("st.global.cs.f64 [%0], %1;" :: "l"(p), "d"(v) : "memory"); }
__device__ __forceinline__ void stcs16(float* p, const float* s) {
    const float4 v = *reinterpret_cast<const float4*>(s);
    asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};" :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
__device__ __forceinline__ void stcs16(double* p, const double* s) {
    const double2 v = *reinterpret_cast<const double2*>(s);
    asm volatile("st.global.cs.v2.f64 [%0], {%1,%2};" :: "l"(p), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(smem_addr(b)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: gives up after about two seconds
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try(b, parity))
        if (gtimer() - t0 > 2000000000ull) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" :: "l"(dst), "r"(smem_addr(src)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
)";

// tile movers of one plan's row layout (macros N, NP, MODE)
const char* kTileFns = R"(
// one thread: whole-tile load (16-byte multiple by TMA, the < 16-byte rest by plain copies)
template <int TS>
__device__ __forceinline__ void bulk_load_tile(const T* __restrict__ x, T* buf, i64 tile, i64 batch, unsigned long long* bar) {
    const T* src = x + tile * (i64)TS * N;
    const int rows = (int)min((i64)TS, batch - tile * (i64)TS);
    const unsigned bytes = (unsigned)(rows * N * sizeof(T));
    const unsigned b16 = bytes & ~15u;
    mbar_expect_tx(bar, b16);
    if (b16) bulk_g2s(buf, src, b16, bar);
    for (unsigned e = b16 / sizeof(T); e < bytes / sizeof(T); ++e) buf[e] = src[e];
}
template <int TS>
__device__ __forceinline__ void bulk_store_tile(const T* buf, T* __restrict__ y, i64 tile, i64 batch) {
    T* dst = y + tile * (i64)TS * N;
    const int rows = (int)min((i64)TS, batch - tile * (i64)TS);
    const unsigned bytes = (unsigned)(rows * N * sizeof(T));
    const unsigned b16 = bytes & ~15u;
    if (b16) bulk_s2g(dst, buf, b16);
    bulk_commit();
    for (unsigned e = b16 / sizeof(T); e < bytes / sizeof(T); ++e) dst[e] = buf[e];
}
template <int THREADS, int TS>
__device__ __forceinline__ void load_tile(const T* __restrict__ x, T* buf, i64 tile, i64 batch) {
    const T* src = x + tile * (i64)TS * N;
    const int rows = (int)min((i64)TS, batch - tile * (i64)TS);
    const int E = rows * N;
    const int tid = threadIdx.x;
#if MODE == 0
    constexpr int PER = 16 / sizeof(T);
    const int E16 = E / PER;
    for (int c = tid; c < E16; c += THREADS) cpa16(buf + c * PER, src + c * PER);
    for (int e = E16 * PER + tid; e < E; e += THREADS) { if (sizeof(T) == 8) cpa8(buf + e, src + e); else cpa4(buf + e, src + e); }
#elif MODE == 1
    const int G = E / 4;
    for (int g = tid; g < G; g += THREADS) { const int t = g / (N / 4), c = g - t * (N / 4); cpa16(buf + t * NP + 4 * c, src + 4 * g); }
#else
    for (int e = tid; e < E; e += THREADS) { const int t = e / N, j = e - t * N; if (sizeof(T) == 8) cpa8(buf + t * NP + j, src + e); else cpa4(buf + t * NP + j, src + e); }
#endif
}
template <int THREADS, int TS>
__device__ __forceinline__ void store_tile(const T* buf, T* __restrict__ y, i64 tile, i64 batch) {
    T* dst = y + tile * (i64)TS * N;
    const int rows = (int)min((i64)TS, batch - tile * (i64)TS);
    const int E = rows * N;
    const int tid = threadIdx.x;
#if MODE == 0
    constexpr int PER = 16 / sizeof(T);
    const int E16 = E / PER;
    for (int c = tid; c < E16; c += THREADS) stcs16(dst + c * PER, buf + c * PER);
    for (int e = E16 * PER + tid; e < E; e += THREADS) stcs(dst + e, buf[e]);
#elif MODE == 1
    const int G = E / 4;
    for (int g = tid; g < G; g += THREADS) { const int t = g / (N / 4), c = g - t * (N / 4); stcs16(dst + 4 * g, buf + t * NP + 4 * c); }
#else
    for (int e = tid; e < E; e += THREADS) { const int t = e / N, j = e - t * N; stcs(dst + e, buf[t * NP + j]); }
#endif
}
)";

const char* kKernelTmpl = R"(
extern "C" __global__ void __launch_bounds__(@THREADS@) @NAME@(const T* __restrict__ x, T* __restrict__ y, i64 batch, int* err) {
    constexpr int THREADS = @THREADS@, RS = @RS@, NBUF = @NBUF@, TS = RS * THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tiles = reinterpret_cast<T*>(smem_raw);
    const int tid = threadIdx.x;
    const i64 ntiles = (batch + TS - 1) / TS;
    i64 tile = blockIdx.x;
    if (tile < ntiles) load_tile<THREADS, TS>(x, tiles, tile, batch);
    commit();
    int cur = 0;
    for (; tile < ntiles; tile += gridDim.x) {
        T* buf = tiles + (NBUF == 2 ? cur * TS * NP : 0);
        const i64 nxt = tile + gridDim.x;
        if (NBUF == 2) {
            if (nxt < ntiles) load_tile<THREADS, TS>(x, tiles + (cur ^ 1) * TS * NP, nxt, batch);
            commit();
            wait1();
        } else {
            wait0();
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < RS; ++s) @BODY@(buf + (tid + s * THREADS) * NP);
        __syncthreads();
        store_tile<THREADS, TS>(buf, y, tile, batch);
        __syncthreads();
        if (NBUF == 2) {
            cur ^= 1;
        } else {
            if (nxt < ntiles) load_tile<THREADS, TS>(x, tiles, nxt, batch);
            commit();
        }
    }
    wait0();
}
)";

// Tiles moved by the TMA engine: one thread issues a bulk copy per tile that
// completes on an mbarrier; after the in-place compute, a bulk store writes
// the tile back.  Waits are bounded (about 2 s), after which the CTA records
// GFT_ERR_TIMEOUT in *err, drains its own bulk copies and returns.
const char* kBulkTmpl = R"(
extern "C" __global__ void __launch_bounds__(@THREADS@) @NAME@(const T* __restrict__ x, T* __restrict__ y, i64 batch, int* err) {
    constexpr int THREADS = @THREADS@, RS = @RS@, NBUF = @NBUF@, TS = RS * THREADS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar[2];
    T* tiles = reinterpret_cast<T*>(smem_raw);
    const int tid = threadIdx.x;
    const i64 ntiles = (batch + TS - 1) / TS;
    i64 tile = blockIdx.x;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phase = 0;
    int cur = 0;
    bool bad = false;
    if (tid == 0 && tile < ntiles) bulk_load_tile<TS>(x, tiles, tile, batch, &mbar[0]);
    for (; tile < ntiles; tile += gridDim.x) {
        const int b = NBUF == 2 ? cur : 0;
        T* buf = tiles + b * TS * NP;
        const i64 nxt = tile + gridDim.x;
        if (NBUF == 2 && tid == 0 && nxt < ntiles) {
            bulk_wait_read0();
            bulk_load_tile<TS>(x, tiles + (cur ^ 1) * TS * NP, nxt, batch, &mbar[cur ^ 1]);
        }
        const bool ok = mbar_wait(&mbar[b], (phase >> b) & 1u);
        phase ^= 1u << b;
        if (__syncthreads_or(!ok)) { bad = true; break; }
#pragma unroll
        for (int s = 0; s < RS; ++s) @BODY@(buf + (tid + s * THREADS) * NP);
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) bulk_store_tile<TS>(buf, y, tile, batch);
        if (NBUF == 2) {
            cur ^= 1;
        } else if (tid == 0 && nxt < ntiles) {
            bulk_wait_read0();
            bulk_load_tile<TS>(x, tiles, nxt, batch, &mbar[0]);
        }
    }
    if (tid == 0) {
        bulk_wait_all();
        if (bad) atomicExch(err, 8);
    }
}
)";

std::string replace_all(std::string s, const std::string& a, const std::string& b) {
    for (size_t pos = s.find(a); pos != std::string::npos; pos = s.find(a, pos + b.size())) s.replace(pos, a.size(), b);
    return s;
}

// per-row straight-line code
std::string gen_bodies(const gft_plan_s& p, bool f64, int mode, bool with_inverse = true) {
    const int n = p.n;
    const char* T = f64 ? "double" : "float";
    const char* FMA = f64 ? "fma" : "fmaf";
    // (leaf, local) for every coefficient position, and the folded matrices
    std::vector<int> leaf_of(n), local_of(n);
    {
        int i = 0;
        for (size_t k = 0; k < p.leaves.size(); ++k)
            for (int c = 0; c < p.leaves[k].m(); ++c, ++i) {
                leaf_of[p.out_pos[i]] = (int)k;
                local_of[p.out_pos[i]] = c;
            }
    }
    auto Mval = [&](int k, int r, int c) {
        const Leaf& lf = p.leaves[k];
        return lf.fold(r, c);
    };
    auto load_row = [&](std::ostringstream& o, const char* v) {
        if (mode == kVec4 && !f64) {
            for (int q = 0; q < n / 4; ++q)
                o << "    { const float4 t = *reinterpret_cast<const float4*>(row + " << 4 * q << "); " << v << 4 * q
                  << " = t.x; " << v << 4 * q + 1 << " = t.y; " << v << 4 * q + 2 << " = t.z; " << v << 4 * q + 3
                  << " = t.w; }\n";
        } else {
            for (int i = 0; i < n; ++i) o << "    " << v << i << " = row[" << i << "];\n";
        }
    };
    std::ostringstream o;
    // ---------------- forward ----------------
    o << "__device__ __noinline__ void body_fwd(" << T << "* __restrict__ row) {\n    " << T << " ";
    for (int i = 0; i < n; ++i) o << "v" << i << (i + 1 < n ? ", " : ";\n");
    load_row(o, "v");
    for (auto& st : p.stages)
        for (auto& pr : st)
            o << "    { const " << T << " a = v" << pr.first << ", b = v" << pr.second << "; v" << pr.first
              << " = a + b; v" << pr.second << " = a - b; }\n";
    auto emit_coeff = [&](std::ostringstream& s, int j, const std::string& dst) {
        const int k = leaf_of[j], c = local_of[j];
        const Leaf& lf = p.leaves[k];
        bool first = true;
        for (int r = 0; r < lf.m(); ++r) {
            const double u = Mval(k, r, c);
            const float uf = (float)u;
            if (f64 ? (u == 0.0) : (uf == 0.0f)) continue;
            if (first) s << "        " << dst << " = v" << lf.labels[r] << " * " << lit(u, f64) << ";\n";
            else s << "        " << dst << " = " << FMA << "(v" << lf.labels[r] << ", " << lit(u, f64) << ", " << dst << ");\n";
            first = false;
        }
        if (first) s << "        " << dst << " = 0;\n";
    };
    if (p.right) {
        // right Haar units: column c of E and of F, then their sum and
        // difference (the 1/sqrt2 is folded into both columns)
        const int m1 = p.leaves[0].m(), pr = (int)p.rpairs.size();
        for (int c = 0; c < pr; ++c) {
            const int jE = p.out_pos[c], jF = p.out_pos[m1 + c];
            o << "    { " << T << " a, b;\n";
            emit_coeff(o, jE, "a");
            emit_coeff(o, jF, "b");
            o << "      row[" << jE << "] = a + b; row[" << jF << "] = a - b; }\n";
        }
        for (int c = pr; c < m1; ++c) {
            const int j = p.out_pos[c];
            o << "    { " << T << " o;\n";
            emit_coeff(o, j, "o");
            o << "      row[" << j << "] = o; }\n";
        }
    } else if (mode == kVec4 && !f64) {
        for (int q = 0; q < n / 4; ++q) {
            o << "    { float o0, o1, o2, o3;\n";
            for (int t = 0; t < 4; ++t) emit_coeff(o, 4 * q + t, "o" + std::to_string(t));
            o << "      *reinterpret_cast<float4*>(row + " << 4 * q << ") = make_float4(o0, o1, o2, o3); }\n";
        }
    } else {
        for (int j = 0; j < n; ++j) {
            o << "    { " << T << " o;\n";
            emit_coeff(o, j, "o");
            o << "      row[" << j << "] = o; }\n";
        }
    }
    o << "}\n";
    if (!with_inverse) return o.str();
    // ---------------- inverse ----------------
    o << "__device__ __noinline__ void body_inv(" << T << "* __restrict__ row) {\n    " << T << " ";
    for (int i = 0; i < n; ++i) o << "v" << i << (i + 1 < n ? ", " : ";\n");
    o << "    " << T << " ";
    for (int i = 0; i < n; ++i) o << "w" << i << (i + 1 < n ? ", " : ";\n");
    load_row(o, "v");
    if (p.right) {   // right Haar units first (each is its own inverse once folded)
        const int m1 = p.leaves[0].m();
        for (int c = 0; c < (int)p.rpairs.size(); ++c) {
            const int jE = p.out_pos[c], jF = p.out_pos[m1 + c];
            o << "    { const " << T << " a = v" << jE << ", b = v" << jF << "; v" << jE << " = a + b; v" << jF
              << " = a - b; }\n";
        }
    }
    {
        int i0 = 0;
        for (size_t k = 0; k < p.leaves.size(); ++k) {
            const Leaf& lf = p.leaves[k];
            const int m = lf.m();
            for (int r = 0; r < m; ++r) {
                const std::string dst = "w" + std::to_string(lf.labels[r]);
                bool first = true;
                for (int c = 0; c < m; ++c) {
                    const double u = Mval((int)k, r, c);
                    if (f64 ? (u == 0.0) : ((float)u == 0.0f)) continue;
                    const int j = p.out_pos[i0 + c];
                    if (first) o << "    " << dst << " = v" << j << " * " << lit(u, f64) << ";\n";
                    else o << "    " << dst << " = " << FMA << "(v" << j << ", " << lit(u, f64) << ", " << dst << ");\n";
                    first = false;
                }
                if (first) o << "    " << dst << " = 0;\n";
            }
            i0 += m;
        }
    }
    for (int s = (int)p.stages.size() - 1; s >= 0; --s)
        for (int q = (int)p.stages[s].size() - 1; q >= 0; --q) {
            auto& pr = p.stages[s][q];
            o << "    { const " << T << " a = w" << pr.first << ", b = w" << pr.second << "; w" << pr.first
              << " = a + b; w" << pr.second << " = a - b; }\n";
        }
    if (mode == kVec4 && !f64) {
        for (int q = 0; q < n / 4; ++q)
            o << "    *reinterpret_cast<float4*>(row + " << 4 * q << ") = make_float4(w" << 4 * q << ", w" << 4 * q + 1
              << ", w" << 4 * q + 2 << ", w" << 4 * q + 3 << ");\n";
    } else {
        for (int i = 0; i < n; ++i) o << "    row[" << i << "] = w" << i << ";\n";
    }
    o << "}\n";
    return o.str();
}

struct Layout {
    int mode, np;
};

Layout row_layout(int n, bool f64) {
    if (n & 1) return {kContig, n};
    if (!f64 && n % 4 == 0) return {kVec4, ((n / 4) & 1) ? n : n + 4};
    return {kPad1, n + 1};
}

std::string kernel_name(bool inverse, int ci) { return std::string(inverse ? "gft_jit_inv_" : "gft_jit_fwd_") + std::to_string(ci); }

std::string gen_module(const gft_plan_s& p, bool f64, const Layout& L, std::vector<int>& cand_ids) {
    std::ostringstream s;
    s << "#define T " << (f64 ? "double" : "float") << "\n#define N " << p.n << "\n#define NP " << L.np
      << "\n#define MODE " << L.mode << "\n";
    s << kHelpers << kTileFns;
    s << gen_bodies(p, f64, L.mode);
    const size_t esz = f64 ? 8 : 4;
    for (int ci = 0; ci < (int)(sizeof(kCands) / sizeof(kCands[0])); ++ci) {
        const Cand& c = kCands[ci];
        const size_t smem = (size_t)c.nbuf * c.rs * c.threads * L.np * esz;
        if (smem > (size_t)kSmemLimitJ) continue;
        if (f64 && ci > 0) break;
        if (c.bulk && L.np != p.n) continue;
        cand_ids.push_back(ci);
        for (int inv = 0; inv < 2; ++inv) {
            std::string k = c.bulk ? kBulkTmpl : kKernelTmpl;
            k = replace_all(k, "@THREADS@", std::to_string(c.threads));
            k = replace_all(k, "@RS@", std::to_string(c.rs));
            k = replace_all(k, "@NBUF@", std::to_string(c.nbuf));
            k = replace_all(k, "@NAME@", kernel_name(inv, ci));
            k = replace_all(k, "@BODY@", inv ? "body_inv" : "body_fwd");
            s << k;
        }
    }
    return s.str();
}

std::vector<char> nvrtc_compile(const std::string& src) {
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "gft_plan.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        fail(GFT_ERR_CUDA, "nvrtcCreateProgram failed");
    const bool verbose = std::getenv("GFT_JIT_VERBOSE") != nullptr;
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device", "--fmad=true",
                          "--ptxas-options=-v"};
    const nvrtcResult r = nvrtcCompileProgram(prog, verbose ? 5 : 4, opts);
    if (verbose && r == NVRTC_SUCCESS) {
        size_t ls = 0;
        nvrtcGetProgramLogSize(prog, &ls);
        std::string log(ls, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        std::fprintf(stderr, "%s\n", log.c_str());
    }
    if (r != NVRTC_SUCCESS) {
        size_t ls = 0;
        nvrtcGetProgramLogSize(prog, &ls);
        std::string log(ls, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        nvrtcDestroyProgram(&prog);
        fail(GFT_ERR_CUDA, "NVRTC compile of the plan kernel failed: " + log.substr(0, 2000));
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    std::vector<char> bin(n);
    nvrtcGetCUBIN(prog, bin.data());
    nvrtcDestroyProgram(&prog);
    return bin;
}

// compiled cubins by source text (identical plans share one compile)
std::mutex g_cache_mu;
std::map<std::string, std::vector<char>>& cubin_cache() {
    static std::map<std::string, std::vector<char>> c;
    return c;
}

}  // namespace

struct JitDir {
    cudaKernel_t k = nullptr;
    int rs = 0, threads = 0, nbuf = 0, per_sm = 0, bulk = 0;
    size_t smem = 0;
    float us = 0.f;
};

struct JitPlan {
    cudaLibrary_t lib32 = nullptr, lib64 = nullptr;
    JitDir d32[2], d64[2];
    JitDir d32_plain[2];   // fastest shape without TMA bulk tiles (zero-copy host buffers)
    int np32 = 0, np64 = 0;
};

bool jit_eligible(const gft_plan_s& p) {
    if (std::getenv("GFT_DISABLE_JIT")) return false;
    if (p.flags & GFT_NO_JIT) return false;
    if (p.n > kJitMaxN) return false;
    return leaf_entries(p) <= kJitMaxLeafEntries;
}

std::string jit_source(const gft_plan_s& p, bool f64) {
    std::vector<int> ids;
    return gen_module(p, f64, row_layout(p.n, f64), ids);
}

static void launch_dir(const JitDir& d, const void* x, void* y, int64_t batch, int* err, cudaStream_t st) {
    const long long ts = (long long)d.rs * d.threads;
    const long long tiles = (batch + ts - 1) / ts;
    const long long grid = std::min<long long>(tiles, (long long)d.per_sm * sm_count());
    long long b = batch;
    void* args[] = {(void*)&x, (void*)&y, (void*)&b, (void*)&err};
    GFT_CUDA(cudaLaunchKernel((const void*)d.k, dim3((unsigned)grid), dim3(d.threads), args, d.smem, st));
}

static void build_precision(gft_plan_s& p, JitPlan& J, bool f64) {
    const Layout L = row_layout(p.n, f64);
    std::vector<int> ids;
    const std::string src = gen_module(p, f64, L, ids);
    std::vector<char> bin;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        auto it = cubin_cache().find(src);
        if (it != cubin_cache().end()) bin = it->second;
    }
    if (bin.empty()) {
        bin = nvrtc_compile(src);
        std::lock_guard<std::mutex> g(g_cache_mu);
        cubin_cache()[src] = bin;
    }
    cudaLibrary_t lib = nullptr;
    GFT_CUDA(cudaLibraryLoadData(&lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    (f64 ? J.lib64 : J.lib32) = lib;
    (f64 ? J.np64 : J.np32) = L.np;
    const size_t esz = f64 ? 8 : 4;
    // autotune: time every compiled launch shape on a batch larger than L2
    const int n = p.n;
    // 192 MB in + 192 MB out: about three times the 129 MB L2, so every shape
    // is timed on HBM traffic, as the transforms of large batches run
    const int64_t tb = std::max<int64_t>(4096, (int64_t)(192ll << 20) / (int64_t)(n * esz));
    void *dx = nullptr, *dy = nullptr;
    GFT_CUDA(cudaMalloc(&dx, tb * n * esz));
    GFT_CUDA(cudaMalloc(&dy, tb * n * esz));
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    try {
        GFT_CUDA(cudaMemset(dx, 0, tb * n * esz));
        GFT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        GFT_CUDA(cudaEventCreate(&e0));
        GFT_CUDA(cudaEventCreate(&e1));
        for (int inv = 0; inv < 2; ++inv) {
            JitDir best;
            for (int ci : ids) {
                const Cand& c = kCands[ci];
                JitDir d;
                GFT_CUDA(cudaLibraryGetKernel(&d.k, lib, kernel_name(inv, ci).c_str()));
                d.rs = c.rs;
                d.threads = c.threads;
                d.nbuf = c.nbuf;
                d.smem = (size_t)c.nbuf * c.rs * c.threads * L.np * esz;
                GFT_CUDA(cudaFuncSetAttribute((const void*)d.k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.smem));
                GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.per_sm, (const void*)d.k, d.threads, d.smem));
                if (d.per_sm < 1) continue;
                d.bulk = c.bulk;
                launch_dir(d, dx, dy, tb, p.dev.d_err, st);
                GFT_CUDA(cudaEventRecord(e0, st));
                for (int r = 0; r < kTuneReps; ++r) launch_dir(d, dx, dy, tb, p.dev.d_err, st);
                GFT_CUDA(cudaEventRecord(e1, st));
                GFT_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                GFT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                d.us = ms * 1000.f / kTuneReps;
                if (!best.k || d.us < best.us) best = d;
                if (!f64 && !c.bulk && (!J.d32_plain[inv].k || d.us < J.d32_plain[inv].us)) J.d32_plain[inv] = d;
            }
            if (!best.k) fail(GFT_ERR_UNSUPPORTED, "no plan-specialised launch shape fits");
            (f64 ? J.d64 : J.d32)[inv] = best;
        }
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        cudaFree(dx);
        cudaFree(dy);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(dx);
    cudaFree(dy);
}

void jit_build(gft_plan_s& p) {
    if (!jit_eligible(p)) return;
    JitPlan* J = new JitPlan;
    try {
        build_precision(p, *J, false);
        if (leaf_entries(p) <= kJitMaxLeafEntries64) build_precision(p, *J, true);
    } catch (...) {
        if (J->lib32) cudaLibraryUnload(J->lib32);
        if (J->lib64) cudaLibraryUnload(J->lib64);
        delete J;
        throw;
    }
    p.jit = J;
}

void jit_free(gft_plan_s& p) {
    if (!p.jit) return;
    JitPlan* J = static_cast<JitPlan*>(p.jit);
    if (J->lib32) cudaLibraryUnload(J->lib32);
    if (J->lib64) cudaLibraryUnload(J->lib64);
    delete J;
    p.jit = nullptr;
}

bool jit_launch(gft_plan_s& p, bool f64, const void* x, void* y, int64_t batch, bool inverse, cudaStream_t st) {
    if (!p.jit || std::getenv("GFT_FORCE_INTERPRETER")) return false;
    JitPlan* J = static_cast<JitPlan*>(p.jit);
    const JitDir& d = (f64 ? J->d64 : J->d32)[inverse ? 1 : 0];
    if (!d.k) return false;
    if (batch > 0) launch_dir(d, x, y, batch, p.dev.d_err, st);
    return true;
}

bool jit_launch_plain(gft_plan_s& p, const float* x, float* y, int64_t batch, cudaStream_t st) {
    if (!p.jit || std::getenv("GFT_FORCE_INTERPRETER")) return false;
    JitPlan* J = static_cast<JitPlan*>(p.jit);
    const JitDir& d = J->d32_plain[0];
    if (!d.k) return false;
    if (batch > 0) launch_dir(d, x, y, batch, p.dev.d_err, st);
    return true;
}

void jit_info(const gft_plan_s& p, int* jit, int* tile, int* threads) {
    *jit = 0;
    *tile = 0;
    *threads = 0;
    if (!p.jit) return;
    const JitPlan* J = static_cast<const JitPlan*>(p.jit);
    *jit = J->d32[0].bulk ? 2 : 1;
    *tile = J->d32[0].rs * J->d32[0].threads;
    *threads = J->d32[0].threads;
}

// ---------------------------------------------------------------------------
// Batch group: the graphs of a mixed batch whose plans are small and shared
// by many entries (the size sweep's deterministic families: thousands of
// skeletons, dozens of cycles or grids of each size).  One module holds the
// straight-line forward body of every such plan (in a namespace of its own,
// with its row layout) and ONE persistent kernel over all their (entry,
// tile) items: a CTA walks a contiguous range of items, switching on the
// item's plan for the tile load, the body and the store, with the next
// item's tile in flight (cp.async) while this one runs.  The bodies are the
// single-plan kernel's, so the outputs agree with the plan's own forward bit
// for bit.
// ---------------------------------------------------------------------------
namespace {

constexpr int kGroupThreads = 128;
constexpr int kGroupMaxN = 64;
constexpr long long kGroupMaxEntries = 2048;
constexpr int kGroupBufFloats = 8448;   // one tile buffer: 33 KB

struct JSegHost {   // same layout as the module's JSeg
    const float* x;
    float* y;
    long long batch;
    long long item0;
    int plan;
    int ts;
};

const char* kGroupKernel = R"(
extern "C" __global__ void __launch_bounds__(128) gft_jit_group(const JSeg* __restrict__ segs, int nseg,
                                                               const i64* __restrict__ range,
                                                               const int* __restrict__ first, int buf_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* tiles = reinterpret_cast<float*>(smem_raw);
    const i64 it0 = range[blockIdx.x], it1 = range[blockIdx.x + 1];
    if (it0 >= it1) return;
    int s = first[blockIdx.x];
    while (s + 1 < nseg && segs[s + 1].item0 <= it0) ++s;
    g_load(segs[s], it0 - segs[s].item0, tiles);
    commit();
    int cur = 0;
    for (i64 it = it0; it < it1; ++it) {
        const JSeg S = segs[s];
        float* buf = tiles + cur * buf_cap;
        int ns = s;
        if (it + 1 < it1) {
            while (ns + 1 < nseg && segs[ns + 1].item0 <= it + 1) ++ns;
            g_load(segs[ns], it + 1 - segs[ns].item0, tiles + (cur ^ 1) * buf_cap);
        }
        commit();
        wait1();
        __syncthreads();
        g_compute(S.plan, buf);
        __syncthreads();
        g_store(S, it - S.item0, buf);
        __syncthreads();
        cur ^= 1;
        s = ns;
    }
    wait0();
}
)";

int group_rs(int np) { return np <= 16 ? 4 : (np <= 33 ? 2 : 1); }

}  // namespace

bool jit_group_eligible(const gft_plan_s& p) {
    if (std::getenv("GFT_DISABLE_JIT")) return false;
    if (!p.has_device || p.n > kGroupMaxN || p.n < 1) return false;
    if (leaf_entries(p) > kGroupMaxEntries) return false;
    const Layout L = row_layout(p.n, false);
    return (size_t)group_rs(L.np) * kGroupThreads * L.np <= (size_t)kGroupBufFloats;
}

struct JitGroup {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t k = nullptr;
    std::vector<JSegHost> segs;    // slot order
    std::vector<int> members;      // slot -> entry index
    JSegHost* d_segs = nullptr;
    long long* d_range = nullptr;
    int* d_first = nullptr;
    long long total_items = 0;
    int grid = 0, buf_cap = 0;
    size_t smem = 0;
    ~JitGroup() {
        if (d_segs) cudaFree(d_segs);
        if (d_range) cudaFree(d_range);
        if (d_first) cudaFree(d_first);
        if (lib) cudaLibraryUnload(lib);
    }
};

std::string jit_group_source(const std::vector<const gft_plan_s*>& uniq) {
    std::ostringstream s;
    s << "#define T float\n#define N 4\n#define NP 4\n#define MODE 0\n" << kHelpers << "#undef N\n#undef NP\n#undef MODE\n";
    std::vector<int> rs(uniq.size()), np(uniq.size());
    for (size_t k = 0; k < uniq.size(); ++k) {
        const gft_plan_s& p = *uniq[k];
        const Layout L = row_layout(p.n, false);
        rs[k] = group_rs(L.np);
        np[k] = L.np;
        s << "namespace jg" << k << " {\n#define N " << p.n << "\n#define NP " << L.np << "\n#define MODE " << L.mode
          << "\n";
        s << kTileFns << gen_bodies(p, false, L.mode, false);
        s << "#undef N\n#undef NP\n#undef MODE\n}\n";
    }
    s << "struct JSeg { const float* x; float* y; i64 batch; i64 item0; int plan; int ts; };\n";
    s << "__device__ __forceinline__ void g_load(const JSeg& S, i64 tile, float* buf) {\n    switch (S.plan) {\n";
    for (size_t k = 0; k < uniq.size(); ++k)
        s << "    case " << k << ": jg" << k << "::load_tile<128, " << rs[k] * kGroupThreads
          << ">(S.x, buf, tile, S.batch); break;\n";
    s << "    }\n}\n";
    s << "__device__ __forceinline__ void g_compute(int plan, float* buf) {\n    switch (plan) {\n";
    for (size_t k = 0; k < uniq.size(); ++k)
        s << "    case " << k << ":\n#pragma unroll\n        for (int r = 0; r < " << rs[k] << "; ++r) jg" << k
          << "::body_fwd(buf + (threadIdx.x + r * 128) * " << np[k] << ");\n        break;\n";
    s << "    }\n}\n";
    s << "__device__ __forceinline__ void g_store(const JSeg& S, i64 tile, const float* buf) {\n    switch (S.plan) {\n";
    for (size_t k = 0; k < uniq.size(); ++k)
        s << "    case " << k << ": jg" << k << "::store_tile<128, " << rs[k] * kGroupThreads
          << ">(buf, S.y, tile, S.batch); break;\n";
    s << "    }\n}\n";
    s << kGroupKernel;
    return s.str();
}

void* jit_group_create(const std::vector<gft_plan_s*>& plans, const std::vector<int64_t>& batches) {
    std::unique_ptr<JitGroup> G(new JitGroup);
    const int k = (int)plans.size();
    std::vector<const gft_plan_s*> uniq;
    std::map<const gft_plan_s*, int> id;
    for (auto* p : plans) {
        if (!jit_group_eligible(*p)) fail(GFT_ERR_UNSUPPORTED, "plan not eligible for the plan-specialised batch group");
        if (!id.count(p)) {
            id[p] = (int)uniq.size();
            uniq.push_back(p);
        }
    }
    const std::string src = jit_group_source(uniq);
    std::vector<char> bin;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        auto it = cubin_cache().find(src);
        if (it != cubin_cache().end()) bin = it->second;
    }
    if (bin.empty()) {
        bin = nvrtc_compile(src);
        std::lock_guard<std::mutex> g(g_cache_mu);
        cubin_cache()[src] = bin;
    }
    GFT_CUDA(cudaLibraryLoadData(&G->lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    GFT_CUDA(cudaLibraryGetKernel(&G->k, G->lib, "gft_jit_group"));
    // slots: plans by decreasing cost per item, the entries of one plan together
    std::vector<double> cpi(uniq.size());
    std::vector<int> ts(uniq.size());
    for (size_t u = 0; u < uniq.size(); ++u) {
        const Layout L = row_layout(uniq[u]->n, false);
        ts[u] = group_rs(L.np) * kGroupThreads;
        G->buf_cap = std::max(G->buf_cap, ts[u] * L.np);
        cpi[u] = (double)ts[u] * (8.0 * uniq[u]->n + 0.1 * (double)leaf_entries(*uniq[u])) + 2000.0;
    }
    G->buf_cap = (G->buf_cap + 3) & ~3;
    G->members.resize(k);
    for (int i = 0; i < k; ++i) G->members[i] = i;
    std::stable_sort(G->members.begin(), G->members.end(), [&](int a, int b) {
        const int ua = id[plans[a]], ub = id[plans[b]];
        return cpi[ua] != cpi[ub] ? cpi[ua] > cpi[ub] : ua < ub;
    });
    std::vector<long long> items;
    double total = 0.0;
    for (int i : G->members) {
        const int u = id[plans[i]];
        JSegHost e{};
        e.batch = batches[i];
        e.item0 = G->total_items;
        e.plan = u;
        e.ts = ts[u];
        items.push_back((batches[i] + ts[u] - 1) / ts[u]);
        G->total_items += items.back();
        total += cpi[u] * (double)items.back();
        G->segs.push_back(e);
    }
    G->smem = 2 * sizeof(float) * (size_t)G->buf_cap;
    GFT_CUDA(cudaFuncSetAttribute((const void*)G->k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G->smem));
    int per_sm = 0;
    GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)G->k, kGroupThreads, G->smem));
    if (per_sm < 1) fail(GFT_ERR_UNSUPPORTED, "plan-specialised batch group does not fit on an SM");
    G->grid = (int)std::max<long long>(1, std::min<long long>(G->total_items, (long long)per_sm * sm_count()));
    // contiguous item ranges of about equal cost, the slot of each range's first item
    std::vector<long long> range(G->grid + 1, G->total_items);
    std::vector<int> first(G->grid, std::max(0, k - 1));
    range[0] = 0;
    first[0] = 0;
    double acc = 0.0;
    int cta = 1;
    for (size_t sl = 0; sl < G->segs.size() && cta < G->grid; ++sl) {
        const double c = cpi[G->segs[sl].plan];
        for (long long t = 0; t < items[sl] && cta < G->grid; ++t) {
            acc += c;
            while (cta < G->grid && acc >= total * cta / G->grid) {
                range[cta] = std::min(G->segs[sl].item0 + t + 1, G->total_items);
                first[cta] = (int)sl;
                ++cta;
            }
        }
    }
    GFT_CUDA(cudaMalloc(&G->d_segs, sizeof(JSegHost) * std::max<size_t>(1, G->segs.size())));
    GFT_CUDA(cudaMalloc(&G->d_range, sizeof(long long) * range.size()));
    GFT_CUDA(cudaMalloc(&G->d_first, sizeof(int) * first.size()));
    GFT_CUDA(cudaMemcpy(G->d_range, range.data(), sizeof(long long) * range.size(), cudaMemcpyHostToDevice));
    GFT_CUDA(cudaMemcpy(G->d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
    return G.release();
}

void jit_group_upload(void* h, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st) {
    JitGroup* G = static_cast<JitGroup*>(h);
    for (size_t sl = 0; sl < G->segs.size(); ++sl) {
        G->segs[sl].x = x[G->members[sl]];
        G->segs[sl].y = y[G->members[sl]];
    }
    if (!G->segs.empty())
        GFT_CUDA(cudaMemcpyAsync(G->d_segs, G->segs.data(), sizeof(JSegHost) * G->segs.size(), cudaMemcpyHostToDevice,
                                 st));
}

void jit_group_launch(void* h, cudaStream_t st) {
    JitGroup* G = static_cast<JitGroup*>(h);
    if (G->total_items == 0) return;
    int nseg = (int)G->segs.size();
    int cap = G->buf_cap;
    void* args[] = {(void*)&G->d_segs, (void*)&nseg, (void*)&G->d_range, (void*)&G->d_first, (void*)&cap};
    GFT_CUDA(cudaLaunchKernel((const void*)G->k, dim3((unsigned)G->grid), dim3(kGroupThreads), args, G->smem, st));
}

void jit_group_free(void* h) { delete static_cast<JitGroup*>(h); }

int jit_group_launches(void* h) { return static_cast<JitGroup*>(h)->total_items > 0 ? 1 : 0; }

int jit_group_tile(void* h, int entry) {
    const JitGroup* G = static_cast<const JitGroup*>(h);
    for (size_t sl = 0; sl < G->segs.size(); ++sl)
        if (G->members[sl] == entry) return G->segs[sl].ts;
    return 0;
}

}  // namespace gft

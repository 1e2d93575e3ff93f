// Device building blocks of the table-driven fast-GFT transform, shared by
// the single-plan kernel (apply.cu) and the mixed-batch kernel (batch.cu).
// See apply.cu for the algorithm and the shared-memory layout.
#pragma once

#include "gft_internal.h"

namespace gft {
namespace core {

template <class T> struct V4;
template <> struct V4<float> {
    float a, b, c, d;
    __device__ __forceinline__ static V4 load(const float* p) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        return {v.x, v.y, v.z, v.w};
    }
};
template <> struct V4<double> {
    double a, b, c, d;
    __device__ __forceinline__ static V4 load(const double* p) {
        const double2 v0 = *reinterpret_cast<const double2*>(p);
        const double2 v1 = *reinterpret_cast<const double2*>(p + 2);
        return {v0.x, v0.y, v1.x, v1.y};
    }
};

struct KArgs {
    const int* ints;
    const void* mats;
    const void* x;
    void* y;
    long long batch;
    int n, np, n_pairs, n_leaves, ints_count;
    int n_pre_pairs;    // pairs before the leaves; the rest are right Haar units on leaf outputs
    int off_labels, off_outpos, off_src, off_desc;
    int mats_smem;      // scalars of one direction's matrices (smem copy)
    int ts;             // signals per tile
    int nbuf;           // input tile buffers (1 or 2)
    int inverse;
    float inv_n;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <class T> __device__ __forceinline__ void cp_async_elem(T* s, const T* g) {
    if constexpr (sizeof(T) == 8) cp_async8(s, g);
    else cp_async4(s, g);
}

// row of flat tile element e, i.e. e / n, via a float reciprocal: exact for
// e < 2^20 because the +0.5 keeps the product at least 0.5/n from an integer
__device__ __forceinline__ int row_of(int e, float inv_n) { return __float2int_rz(((float)e + 0.5f) * inv_n); }

template <class T, int THREADS>
__device__ __forceinline__ void issue_tile_load(const KArgs& a, const int* src_slot, T* buf, long long tile) {
    const T* src = reinterpret_cast<const T*>(a.x) + tile * (long long)a.ts * a.n;
    const long long rows = min((long long)a.ts, a.batch - tile * (long long)a.ts);
    const int E = (int)rows * a.n;
    const int tid = threadIdx.x;
    if (a.inverse) {  // coefficient j of signal t goes to slot src[j] of row t
        for (int e = tid; e < E; e += THREADS) {
            const int t = row_of(e, a.inv_n);
            cp_async_elem(buf + t * a.np + src_slot[e - t * a.n], src + e);
        }
    } else if (a.np == a.n) {  // odd n: the tile keeps the global layout; 16 B per copy
        constexpr int PER = 16 / sizeof(T);
        const int E16 = E / PER;
        for (int c = tid; c < E16; c += THREADS) cp_async16(buf + c * PER, src + c * PER);
        for (int e = E16 * PER + tid; e < E; e += THREADS) cp_async_elem(buf + e, src + e);
    } else {
        for (int e = tid; e < E; e += THREADS) {
            const int t = row_of(e, a.inv_n);
            cp_async_elem(buf + t * a.np + (e - t * a.n), src + e);
        }
    }
}

template <class T> struct Vec4Store;
template <> struct Vec4Store<float> {
    __device__ __forceinline__ static void st(float* p, float a, float b, float c, float d) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
    }
};
template <> struct Vec4Store<double> {
    __device__ __forceinline__ static void st(double* p, double a, double b, double c, double d) {
        __stcs(reinterpret_cast<double2*>(p), make_double2(a, b));
        __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(c, d));
    }
};

// Store a tile: forward reads coefficient j of row t from slot src[j];
// inverse stores the rows as they are.  Four consecutive outputs per
// thread and 16-byte-aligned vector stores (the tile start is a multiple of
// 4 elements because TS is a multiple of 4).
template <class T, int THREADS>
__device__ __forceinline__ void store_tile(const KArgs& a, const int* src_slot, const T* buf, long long tile) {
    T* dst = reinterpret_cast<T*>(a.y) + tile * (long long)a.ts * a.n;
    const long long rows = min((long long)a.ts, a.batch - tile * (long long)a.ts);
    const int E = (int)rows * a.n;
    const int E4 = E / 4;
    const int tid = threadIdx.x;
    const bool fwd = !a.inverse;
    for (int c = tid; c < E4; c += THREADS) {
        T v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = 4 * c + q;
            const int t = row_of(e, a.inv_n);
            const int j = e - t * a.n;
            v[q] = buf[t * a.np + (fwd ? src_slot[j] : j)];
        }
        Vec4Store<T>::st(dst + 4 * c, v[0], v[1], v[2], v[3]);
    }
    for (int e = E4 * 4 + tid; e < E; e += THREADS) {
        const int t = row_of(e, a.inv_n);
        const int j = e - t * a.n;
        __stcs(dst + e, buf[t * a.np + (fwd ? src_slot[j] : j)]);
    }
}

// In place for the RS signals this thread owns: with v_r = row[idx[r]],
// row[idx[c]] = sum_r v_r * M[r][c] (c < m).  M is BK x BK row-major in
// shared memory, zero beyond m.
template <class T, int BK, int RS, int THREADS>
__device__ __forceinline__ void leaf_product(T* tile, int np, const int* idx, const T* M, int m) {
    const int tid = threadIdx.x;
    T xr[RS][BK];
#pragma unroll
    for (int r = 0; r < BK; ++r) {
        if (r < m) {
            const int g = idx[r];
#pragma unroll
            for (int s = 0; s < RS; ++s) xr[s][r] = tile[(tid + s * THREADS) * np + g];
        } else {
#pragma unroll
            for (int s = 0; s < RS; ++s) xr[s][r] = T(0);
        }
    }
    for (int c0 = 0; c0 < m; c0 += 4) {
        T acc[RS][4];
#pragma unroll
        for (int s = 0; s < RS; ++s) acc[s][0] = acc[s][1] = acc[s][2] = acc[s][3] = T(0);
#pragma unroll
        for (int r = 0; r < BK; ++r) {
            if (r < m) {
                const V4<T> u = V4<T>::load(M + r * BK + c0);
#pragma unroll
                for (int s = 0; s < RS; ++s) {
                    acc[s][0] = fma(xr[s][r], u.a, acc[s][0]);
                    acc[s][1] = fma(xr[s][r], u.b, acc[s][1]);
                    acc[s][2] = fma(xr[s][r], u.c, acc[s][2]);
                    acc[s][3] = fma(xr[s][r], u.d, acc[s][3]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (c0 + j < m) {
                const int o = idx[c0 + j];
#pragma unroll
                for (int s = 0; s < RS; ++s) tile[(tid + s * THREADS) * np + o] = acc[s][j];
            }
        }
    }
}

template <class T, int RS, int THREADS>
__device__ __forceinline__ void leaf_dispatch(int bk, T* tile, int np, const int* idx, const T* M, int m) {
    if (bk == 4) leaf_product<T, 4, RS, THREADS>(tile, np, idx, M, m);
    else if (bk == 8) leaf_product<T, 8, RS, THREADS>(tile, np, idx, M, m);
    else if (bk == 16) leaf_product<T, 16, RS, THREADS>(tile, np, idx, M, m);
    else {
        if constexpr (RS <= 2) {
            if (bk == 24) leaf_product<T, 24, RS, THREADS>(tile, np, idx, M, m);
            else if (bk == 32) leaf_product<T, 32, RS, THREADS>(tile, np, idx, M, m);
        }
        if constexpr (RS == 1) {
            if (bk == 48) leaf_product<T, 48, 1, THREADS>(tile, np, idx, M, m);
            else if (bk == 64) leaf_product<T, 64, 1, THREADS>(tile, np, idx, M, m);
        }
    }
}

// Haar units p0, p0 + step, ... (count of them) on the RS rows of this thread.
template <class T, int RS, int THREADS>
__device__ __forceinline__ void haar_units(T* tile, int np, const int* pairs, int p0, int count, int step) {
    const int tid = threadIdx.x;
    for (int q = 0; q < count; ++q) {
        const int p = p0 + q * step;
        const int i = pairs[2 * p], j = pairs[2 * p + 1];
#pragma unroll
        for (int s = 0; s < RS; ++s) {
            T* row = tile + (tid + s * THREADS) * np;
            const T u = row[i], v = row[j];
            row[i] = u + v;
            row[j] = u - v;
        }
    }
}

// One tile in place for the RS signals of every thread.  Forward: left
// stages, leaf products, right Haar units (bipartite plans).  Inverse: the
// right units, leaf products, left stages in reverse (every unit is its own
// inverse once the 1/sqrt2 factors are folded into the leaf matrices).
template <class T, int RS, int THREADS>
__device__ __forceinline__ void compute_tile(const KArgs& a, const int* ints, const T* mats, T* tile) {
    const int np = a.np;
    const int* pairs = ints;
    const int* labels = ints + a.off_labels;
    const int* desc = ints + a.off_desc;
    const int pre = a.n_pre_pairs, post = a.n_pairs - a.n_pre_pairs;
    if (!a.inverse) haar_units<T, RS, THREADS>(tile, np, pairs, 0, pre, 1);
    else haar_units<T, RS, THREADS>(tile, np, pairs, a.n_pairs - 1, post, -1);
    for (int k = 0; k < a.n_leaves; ++k) {
        const int* d = desc + kLeafDesc * k;
        leaf_dispatch<T, RS, THREADS>(d[1], tile, np, labels + d[2], mats + d[4], d[0]);
    }
    if (!a.inverse) haar_units<T, RS, THREADS>(tile, np, pairs, pre, post, 1);
    else haar_units<T, RS, THREADS>(tile, np, pairs, pre - 1, pre, -1);
}


}  // namespace core
}  // namespace gft

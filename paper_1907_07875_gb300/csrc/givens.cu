// Layered Givens rotations (Eq. 1, Fig. 1): the learned surrogate that
// stands in for a dense GFT on nearly symmetric graphs.
//
//   forward:  per stage s and pair k = (p, q) with angle theta:
//             (y_p, y_q) = (c x_p - s x_q, s x_p + c x_q)
//   backward: from the forward OUTPUT y and the loss gradient g = dL/dy,
//             stage by stage in reverse:
//               dL/dtheta += -g_p y_q + g_q y_p        (since dy_p = -y_q dtheta,
//                                                       dy_q = y_p dtheta)
//               x = G^T y (recover the stage input, no stored activations)
//               g <- G^T g
//
// One thread owns one signal (its row lives in shared memory with an odd
// stride, so lanes hit distinct banks).  Angle gradients: each warp reduces
// its 32 contributions with shuffles into a per-warp shared array (no
// atomics), the CTA sums its warps in fixed order into a per-CTA row of a
// device scratch buffer, and a second kernel sums the rows in fixed order:
// the result is deterministic.
#include <algorithm>
#include <memory>
#include <vector>

#include "gft_internal.h"

struct gft_givens_s {
    int n = 0, S = 0;
    int xor_log2 = 0;              // > 0: butterfly wiring (stage t pairs i, i ^ 2^(t mod log2 n)), n <= 64
    int brick = 0;                 // 1: neighbour wiring (even stages (2k, 2k+1), odd (2k+1, 2k+2) and (n-1, 0))
    int* d_pairs = nullptr;        // S * n/2 * 2
    float* d_partials = nullptr;   // grid * S * n/2 (scratch for the backward pass)
    int partial_rows = 0;
    ~gft_givens_s() {
        if (d_pairs) cudaFree(d_pairs);
        if (d_partials) cudaFree(d_partials);
    }
};

namespace gft {

namespace {

constexpr int kGivThreads = 128;
constexpr int kSmemLimitG = 232448;

__device__ __forceinline__ int row_of_g(int e, float inv_n) { return __float2int_rz(((float)e + 0.5f) * inv_n); }

// coalesced tile load of `rows` signals into smem rows of stride np
__device__ __forceinline__ void load_rows(const float* src, float* dst, int rows, int n, int np, float inv_n) {
    const int E = rows * n;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int t = row_of_g(e, inv_n);
        dst[t * np + (e - t * n)] = src[e];
    }
}

__device__ __forceinline__ void store_rows(const float* src, float* dst, int rows, int n, int np, float inv_n) {
    const int E = rows * n;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int t = row_of_g(e, inv_n);
        dst[e] = src[t * np + (e - t * n)];
    }
}

struct GArgs {
    const int* pairs;
    const float* theta;
    const float* x;     // forward: input; backward: forward output y
    const float* g;     // backward: dL/dy
    float* y;           // forward: output; backward: dL/dx
    float* partials;    // backward: [gridDim.x][A]
    long long batch;
    int n, np, S, A;    // A = S * n/2 angles
    float inv_n;
};

__global__ void __launch_bounds__(kGivThreads) givens_fwd_kernel(GArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    int* pr = reinterpret_cast<int*>(sm);                 // 2A
    float* cs = reinterpret_cast<float*>(pr + 2 * a.A);   // 2A
    float* tile = cs + 2 * a.A;                           // kGivThreads * np
    for (int i = threadIdx.x; i < a.A; i += blockDim.x) {
        pr[2 * i] = a.pairs[2 * i];
        pr[2 * i + 1] = a.pairs[2 * i + 1];
        float s, c;
        sincosf(a.theta[i], &s, &c);
        cs[2 * i] = c;
        cs[2 * i + 1] = s;
    }
    const long long n_tiles = (a.batch + kGivThreads - 1) / kGivThreads;
    for (long long tl = blockIdx.x; tl < n_tiles; tl += gridDim.x) {
        const int rows = (int)min((long long)kGivThreads, a.batch - tl * kGivThreads);
        __syncthreads();
        load_rows(a.x + tl * kGivThreads * a.n, tile, rows, a.n, a.np, a.inv_n);
        __syncthreads();
        if ((int)threadIdx.x < rows) {
            float* r = tile + threadIdx.x * a.np;
            for (int i = 0; i < a.A; ++i) {
                const int p = pr[2 * i], q = pr[2 * i + 1];
                const float c = cs[2 * i], s = cs[2 * i + 1];
                const float xp = r[p], xq = r[q];
                r[p] = fmaf(c, xp, -s * xq);
                r[q] = fmaf(s, xp, c * xq);
            }
        }
        __syncthreads();
        store_rows(tile, a.y + tl * kGivThreads * a.n, rows, a.n, a.np, a.inv_n);
    }
}

// Forward pass for the butterfly wiring (the surrogate's default): stage t
// pairs i with i ^ 2^(t mod log2 N) in ascending order of the lower index,
// so every index is a compile-time constant once the log2 N stages of a
// round are unrolled.  Each thread keeps its signal in registers; per
// rotation it reads one (cos, sin) pair (a shared-memory broadcast) and
// issues two multiplies and two FMAs -- the same arithmetic, in the same
// order, as the general kernel.  Tiles of 128 signals move with 16-byte
// cp.async copies into rows of stride N + 4 floats (16-byte aligned, and the
// 16-byte row reads of consecutive lanes hit distinct banks).
// The neighbour ("brick") wiring of the learned correction runs in the same
// kernel with BRICK = true: even stages pair (2k, 2k+1), odd stages
// (2k+1, 2k+2) and close the ring with (N-1, 0); a round is two stages.
template <int N, bool BRICK>
__global__ void __launch_bounds__(kGivThreads) givens_fwd_xor_kernel(GArgs a) {
    constexpr int LG = BRICK ? 2 : N == 4 ? 2 : N == 8 ? 3 : N == 16 ? 4 : N == 32 ? 5 : 6;
    constexpr int H = N / 2;
    constexpr int NP = N + 4;
    extern __shared__ __align__(16) unsigned char sm[];
    float2* cs = reinterpret_cast<float2*>(sm);                                    // A
    float* tile = reinterpret_cast<float*>(sm + ((sizeof(float2) * a.A + 15) & ~size_t(15)));   // 128 x NP
    for (int i = threadIdx.x; i < a.A; i += blockDim.x) {
        float sn, c;
        sincosf(a.theta[i], &sn, &c);
        cs[i] = make_float2(c, sn);
    }
    const long long n_tiles = (a.batch + kGivThreads - 1) / kGivThreads;
    for (long long tl = blockIdx.x; tl < n_tiles; tl += gridDim.x) {
        const int rows = (int)min((long long)kGivThreads, a.batch - tl * kGivThreads);
        const float* src = a.x + tl * kGivThreads * N;
        __syncthreads();   // previous tile stored, angles written
        for (int c = threadIdx.x; c < rows * (N / 4); c += kGivThreads) {
            const int t = c / (N / 4), k = c - t * (N / 4);
            const unsigned d = (unsigned)__cvta_generic_to_shared(tile + t * NP + 4 * k);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + 4 * c) : "memory");
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if ((int)threadIdx.x < rows) {
            float* row = tile + threadIdx.x * NP;
            float r[N];
#pragma unroll
            for (int q = 0; q < N / 4; ++q) {
                const float4 v = reinterpret_cast<const float4*>(row)[q];
                r[4 * q] = v.x;
                r[4 * q + 1] = v.y;
                r[4 * q + 2] = v.z;
                r[4 * q + 3] = v.w;
            }
            for (int s0 = 0; s0 < a.S; s0 += LG) {
#pragma unroll
                for (int b = 0; b < LG; ++b) {
                    if (s0 + b < a.S) {
                        const float2* st = cs + (s0 + b) * H;
                        constexpr int dummy = 0;
                        (void)dummy;
#pragma unroll
                        for (int k = 0; k < H; ++k) {
                            const int lo = BRICK ? (b == 0 ? 2 * k : (k + 1 < H ? 2 * k + 1 : N - 1))
                                                 : ((k >> b) << (b + 1)) | (k & ((1 << b) - 1));
                            const int hi = BRICK ? (b == 0 ? 2 * k + 1 : (k + 1 < H ? 2 * k + 2 : 0)) : lo | (1 << b);
                            const float2 w = st[k];
                            const float xp = r[lo], xq = r[hi];
                            r[lo] = fmaf(w.x, xp, -w.y * xq);
                            r[hi] = fmaf(w.y, xp, w.x * xq);
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < N / 4; ++q)
                reinterpret_cast<float4*>(row)[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        }
        __syncthreads();
        float* dst = a.y + tl * kGivThreads * N;
        for (int c = threadIdx.x; c < rows * (N / 4); c += kGivThreads) {
            const int t = c / (N / 4), k = c - t * (N / 4);
            __stcs(reinterpret_cast<float4*>(dst) + c, *reinterpret_cast<const float4*>(tile + t * NP + 4 * k));
        }
    }
}

__global__ void __launch_bounds__(kGivThreads) givens_bwd_kernel(GArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr int W = kGivThreads / 32;
    int* pr = reinterpret_cast<int*>(sm);                 // 2A
    float* cs = reinterpret_cast<float*>(pr + 2 * a.A);   // 2A
    float* acc = cs + 2 * a.A;                            // W * A (per-warp sums)
    float* ty = acc + W * a.A;                            // kGivThreads * np
    float* tg = ty + kGivThreads * a.np;                  // kGivThreads * np
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < a.A; i += blockDim.x) {
        pr[2 * i] = a.pairs[2 * i];
        pr[2 * i + 1] = a.pairs[2 * i + 1];
        float s, c;
        sincosf(a.theta[i], &s, &c);
        cs[2 * i] = c;
        cs[2 * i + 1] = s;
    }
    for (int i = threadIdx.x; i < W * a.A; i += blockDim.x) acc[i] = 0.f;
    const long long n_tiles = (a.batch + kGivThreads - 1) / kGivThreads;
    for (long long tl = blockIdx.x; tl < n_tiles; tl += gridDim.x) {
        const int rows = (int)min((long long)kGivThreads, a.batch - tl * kGivThreads);
        __syncthreads();
        load_rows(a.x + tl * kGivThreads * a.n, ty, rows, a.n, a.np, a.inv_n);
        load_rows(a.g + tl * kGivThreads * a.n, tg, rows, a.n, a.np, a.inv_n);
        __syncthreads();
        const bool live = (int)threadIdx.x < rows;
        float* ry = ty + threadIdx.x * a.np;
        float* rg = tg + threadIdx.x * a.np;
        for (int i = a.A - 1; i >= 0; --i) {
            const int p = pr[2 * i], q = pr[2 * i + 1];
            const float c = cs[2 * i], s = cs[2 * i + 1];
            float d = 0.f;
            if (live) {
                const float yp = ry[p], yq = ry[q], gp = rg[p], gq = rg[q];
                d = gq * yp - gp * yq;
                ry[p] = c * yp + s * yq;     // x = G^T y
                ry[q] = -s * yp + c * yq;
                rg[p] = c * gp + s * gq;     // g <- G^T g
                rg[q] = -s * gp + c * gq;
            }
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if (lane == 0) acc[warp * a.A + i] += d;
        }
        __syncthreads();
        store_rows(tg, a.y + tl * kGivThreads * a.n, rows, a.n, a.np, a.inv_n);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.A; i += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < W; ++w) s += acc[w * a.A + i];
        a.partials[(long long)blockIdx.x * a.A + i] = s;
    }
}

__global__ void givens_reduce_kernel(const float* partials, int rows, int A, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += partials[(long long)r * A + i];
    out[i] = s;
}

size_t fwd_smem(int A, int np) { return sizeof(int) * 2 * A + sizeof(float) * (2 * A + (size_t)kGivThreads * np); }
size_t bwd_smem(int A, int np) {
    return sizeof(int) * 2 * A + sizeof(float) * (2 * A + (size_t)(kGivThreads / 32) * A + 2 * (size_t)kGivThreads * np);
}

void check_io_g(const void* a, const void* b, int64_t batch) {
    if (batch < 0) fail(GFT_ERR_INVALID_ARG, "batch < 0");
    if (batch == 0) return;
    if (!a || !b) fail(GFT_ERR_INVALID_ARG, "NULL pointer");
    if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u)
        fail(GFT_ERR_MISALIGNED, "pointers must be 16-byte aligned");
}

}  // namespace

// exported through abi_givens below
void givens_forward(gft_givens_s& g, const float* theta, const float* x, float* y, int64_t batch, cudaStream_t st) {
    if (batch == 0) return;
    if (g.xor_log2 || g.brick) {
        GArgs a{};
        a.theta = theta;
        a.x = x;
        a.y = y;
        a.batch = batch;
        a.n = g.n;
        a.S = g.S;
        a.A = g.S * g.n / 2;
        void (*fn)(GArgs);
        if (g.brick)
            fn = g.n == 4 ? givens_fwd_xor_kernel<4, true> : g.n == 8 ? givens_fwd_xor_kernel<8, true>
               : g.n == 16 ? givens_fwd_xor_kernel<16, true> : g.n == 32 ? givens_fwd_xor_kernel<32, true>
               : givens_fwd_xor_kernel<64, true>;
        else
            fn = g.n == 4 ? givens_fwd_xor_kernel<4, false> : g.n == 8 ? givens_fwd_xor_kernel<8, false>
               : g.n == 16 ? givens_fwd_xor_kernel<16, false> : g.n == 32 ? givens_fwd_xor_kernel<32, false>
               : givens_fwd_xor_kernel<64, false>;
        const size_t smem = ((sizeof(float2) * a.A + 15) & ~size_t(15)) + sizeof(float) * kGivThreads * (g.n + 4);
        GFT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kGivThreads, smem));
        const long long tiles = (batch + kGivThreads - 1) / kGivThreads;
        const long long grid = std::min<long long>(tiles, (long long)std::max(1, per_sm) * sm_count());
        fn<<<(unsigned)grid, kGivThreads, smem, st>>>(a);
        GFT_CUDA(cudaGetLastError());
        return;
    }
    GArgs a{};
    a.pairs = g.d_pairs;
    a.theta = theta;
    a.x = x;
    a.y = y;
    a.batch = batch;
    a.n = g.n;
    a.np = g.n | 1;
    a.S = g.S;
    a.A = g.S * g.n / 2;
    a.inv_n = 1.0f / g.n;
    const size_t smem = fwd_smem(a.A, a.np);
    if (smem > (size_t)kSmemLimitG) fail(GFT_ERR_UNSUPPORTED, "Givens network too large for shared memory");
    GFT_CUDA(cudaFuncSetAttribute(givens_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, givens_fwd_kernel, kGivThreads, smem));
    const long long tiles = (batch + kGivThreads - 1) / kGivThreads;
    const long long grid = std::min<long long>(tiles, (long long)std::max(1, per_sm) * sm_count());
    givens_fwd_kernel<<<(unsigned)grid, kGivThreads, smem, st>>>(a);
    GFT_CUDA(cudaGetLastError());
}

void givens_backward(gft_givens_s& g, const float* theta, const float* y, const float* gy, float* gx,
                     float* gtheta, int64_t batch, cudaStream_t st) {
    const int A = g.S * g.n / 2;
    if (batch == 0) {
        GFT_CUDA(cudaMemsetAsync(gtheta, 0, sizeof(float) * A, st));
        return;
    }
    GArgs a{};
    a.pairs = g.d_pairs;
    a.theta = theta;
    a.x = y;
    a.g = gy;
    a.y = gx;
    a.batch = batch;
    a.n = g.n;
    a.np = g.n | 1;
    a.S = g.S;
    a.A = A;
    a.inv_n = 1.0f / g.n;
    const size_t smem = bwd_smem(A, a.np);
    if (smem > (size_t)kSmemLimitG) fail(GFT_ERR_UNSUPPORTED, "Givens network too large for the backward kernel");
    GFT_CUDA(cudaFuncSetAttribute(givens_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, givens_bwd_kernel, kGivThreads, smem));
    const long long tiles = (batch + kGivThreads - 1) / kGivThreads;
    const int grid = (int)std::min<long long>(tiles, (long long)std::max(1, per_sm) * sm_count());
    if (g.partial_rows < grid) {
        if (g.d_partials) cudaFree(g.d_partials);
        g.d_partials = nullptr;
        g.partial_rows = 0;
        GFT_CUDA(cudaMalloc(&g.d_partials, sizeof(float) * (size_t)grid * A));
        g.partial_rows = grid;
    }
    a.partials = g.d_partials;
    givens_bwd_kernel<<<grid, kGivThreads, smem, st>>>(a);
    GFT_CUDA(cudaGetLastError());
    givens_reduce_kernel<<<(A + 127) / 128, 128, 0, st>>>(g.d_partials, grid, A, gtheta);
    GFT_CUDA(cudaGetLastError());
}

}  // namespace gft

using namespace gft;

namespace gft {
template <class F> gft_status guard_g(F&& f) {
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
}  // namespace gft

extern "C" {

gft_status gft_givens_create(int32_t n, int32_t n_stages, const int32_t* pairs, gft_givens_t* out) {
    return guard_g([&] {
        if (!out || !pairs) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        if (n < 2 || n > 1024 || (n & 1)) fail(GFT_ERR_INVALID_ARG, "n must be even, 2..1024");
        if (n_stages < 1 || n_stages > 64) fail(GFT_ERR_INVALID_ARG, "n_stages must be 1..64");
        const int half = n / 2;
        std::vector<int> seen(n);
        for (int s = 0; s < n_stages; ++s) {
            std::fill(seen.begin(), seen.end(), 0);
            for (int k = 0; k < half; ++k) {
                const int p = pairs[(size_t)(s * half + k) * 2], q = pairs[(size_t)(s * half + k) * 2 + 1];
                if (p < 0 || p >= n || q < 0 || q >= n || p == q || seen[p] || seen[q])
                    fail(GFT_ERR_INVALID_ARG, "stage " + std::to_string(s) + " is not a perfect matching");
                seen[p] = seen[q] = 1;
            }
        }
        std::unique_ptr<gft_givens_s> g(new gft_givens_s);
        g->n = n;
        g->S = n_stages;
        int lg = 0;
        while ((1 << lg) < n) ++lg;
        if ((1 << lg) == n && n >= 4 && n <= 64) {
            bool ok = true;
            for (int s = 0; s < n_stages && ok; ++s) {
                const int b = s % lg;
                for (int k = 0; k < half && ok; ++k) {
                    const int lo = ((k >> b) << (b + 1)) | (k & ((1 << b) - 1));
                    ok = pairs[(size_t)(s * half + k) * 2] == lo && pairs[(size_t)(s * half + k) * 2 + 1] == (lo | (1 << b));
                }
            }
            if (ok) g->xor_log2 = lg;
            bool br = !ok;
            for (int s = 0; s < n_stages && br; ++s)
                for (int k = 0; k < half && br; ++k) {
                    const int lo = (s & 1) == 0 ? 2 * k : (k + 1 < half ? 2 * k + 1 : n - 1);
                    const int hi = (s & 1) == 0 ? 2 * k + 1 : (k + 1 < half ? 2 * k + 2 : 0);
                    br = pairs[(size_t)(s * half + k) * 2] == lo && pairs[(size_t)(s * half + k) * 2 + 1] == hi;
                }
            if (br) g->brick = 1;
        }
        const size_t cnt = (size_t)n_stages * half * 2;
        GFT_CUDA(cudaMalloc(&g->d_pairs, sizeof(int) * cnt));
        GFT_CUDA(cudaMemcpy(g->d_pairs, pairs, sizeof(int) * cnt, cudaMemcpyHostToDevice));
        *out = g.release();
    });
}

gft_status gft_givens_destroy(gft_givens_t g) {
    return guard_g([&] { delete g; });
}

gft_status gft_givens_forward(gft_givens_t g, const float* theta, const float* x, float* y, int64_t batch,
                              gft_stream_t stream) {
    return guard_g([&] {
        if (!g || !theta) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        check_io_g(x, y, batch);
        givens_forward(*g, theta, x, y, batch, reinterpret_cast<cudaStream_t>(stream));
    });
}

gft_status gft_givens_backward(gft_givens_t g, const float* theta, const float* y, const float* gy, float* gx,
                               float* gtheta, int64_t batch, gft_stream_t stream) {
    return guard_g([&] {
        if (!g || !theta || !gtheta) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        check_io_g(y, gy, batch);
        check_io_g(gx, gy, batch);
        givens_backward(*g, theta, y, gy, gx, gtheta, batch, reinterpret_cast<cudaStream_t>(stream));
    });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free backward pass of the Givens layers.
//
// Some callers cannot allocate device memory while they run: programs that
// hand every byte of the GPU to their own memory pool or a fixed budget,
// real-time training or serving loops that must neither wait for nor risk a
// failed allocation in the middle of a step, and hosts that reach this
// library through a thin C interface with no allocator of their own.
// gft_givens_backward_noalloc serves them.  It takes the pair table from
// host memory and everything else from caller-owned device buffers, and
// keeps its only scratch -- the pair table copy and one row of partial angle
// sums per CTA -- in a fixed array compiled into this library.  That array
// (kNoAllocScratchBytes) occupies device memory on every GPU that loads the
// library until the process exits.  Host code cannot use the array's name
// as a device address, so its address is looked up once per device with
// cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
#include <mutex>

namespace gft {
namespace {

constexpr size_t kNoAllocScratchBytes = 4u << 20;  // 4 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the fixed scratch on the current device; the first call
// on each device performs the lookup.
void* noalloc_scratch() {
    int dev = 0;
    GFT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) fail(GFT_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(GFT_ERR_CUDA, std::string("cudaGetSymbolAddress of the fixed scratch failed: ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    return g_noalloc_addr[dev];
}

}  // namespace
}  // namespace gft

extern "C" gft_status gft_givens_backward_noalloc(int32_t n, int32_t n_stages, const int32_t* pairs,
                                                  const float* theta, const float* y, const float* gy, float* gx,
                                                  float* gtheta, int64_t batch, gft_stream_t stream) {
    return guard_g([&] {
        if (!pairs || !theta || !gtheta) fail(GFT_ERR_INVALID_ARG, "NULL argument");
        if (n < 2 || n > 1024 || (n & 1)) fail(GFT_ERR_INVALID_ARG, "n must be even, 2..1024");
        if (n_stages < 1 || n_stages > 64) fail(GFT_ERR_INVALID_ARG, "n_stages must be 1..64");
        check_io_g(y, gy, batch);
        check_io_g(gx, gy, batch);
        const int half = n / 2;
        bool seen[1024];
        for (int s = 0; s < n_stages; ++s) {
            for (int i = 0; i < n; ++i) seen[i] = false;
            for (int k = 0; k < half; ++k) {
                const int p = pairs[(size_t)(s * half + k) * 2], q = pairs[(size_t)(s * half + k) * 2 + 1];
                if (p < 0 || p >= n || q < 0 || q >= n || p == q || seen[p] || seen[q])
                    fail(GFT_ERR_INVALID_ARG, "stage " + std::to_string(s) + " is not a perfect matching");
                seen[p] = seen[q] = true;
            }
        }
        const int A = n_stages * half;
        const size_t pair_bytes = ((size_t)n_stages * n * sizeof(int) + 255) & ~size_t(255);
        const size_t row_bytes = (size_t)A * sizeof(float);
        if (pair_bytes + row_bytes > kNoAllocScratchBytes)
            fail(GFT_ERR_INVALID_ARG, "network needs more than the fixed 4 MiB scratch");
        const long long rows_cap = (long long)((kNoAllocScratchBytes - pair_bytes) / row_bytes);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        unsigned char* scratch = static_cast<unsigned char*>(noalloc_scratch());
        // the pair table region is rewritten by every call
        GFT_CUDA(cudaMemcpyAsync(scratch, pairs, (size_t)n_stages * n * sizeof(int), cudaMemcpyHostToDevice, st));
        if (batch == 0) {
            GFT_CUDA(cudaMemsetAsync(gtheta, 0, row_bytes, st));
            return;
        }
        GArgs a{};
        a.pairs = reinterpret_cast<const int*>(scratch);
        a.theta = theta;
        a.x = y;
        a.g = gy;
        a.y = gx;
        a.partials = reinterpret_cast<float*>(scratch + pair_bytes);
        a.batch = batch;
        a.n = n;
        a.np = n | 1;
        a.S = n_stages;
        a.A = A;
        a.inv_n = 1.0f / n;
        const size_t smem = bwd_smem(A, a.np);
        if (smem > (size_t)kSmemLimitG) fail(GFT_ERR_UNSUPPORTED, "Givens network too large for the backward kernel");
        GFT_CUDA(cudaFuncSetAttribute(givens_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, givens_bwd_kernel, kGivThreads, smem));
        const long long tiles = (batch + kGivThreads - 1) / kGivThreads;
        // every CTA overwrites its whole partial row, and the reduction reads
        // only the rows of this call: nothing in the scratch needs clearing.
        // rows_cap is a guard only: the shared-memory limit above keeps A
        // below about 3.6k angles, so at least 280 rows fit in the 4 MiB,
        // more than the resident CTAs of the whole GPU at these shapes.
        const int grid = (int)std::min(std::min<long long>(tiles, (long long)std::max(1, per_sm) * sm_count()), rows_cap);
        givens_bwd_kernel<<<grid, kGivThreads, smem, st>>>(a);
        GFT_CUDA(cudaGetLastError());
        givens_reduce_kernel<<<(A + 127) / 128, 128, 0, st>>>(a.partials, grid, A, gtheta);
        GFT_CUDA(cudaGetLastError());
    });
}

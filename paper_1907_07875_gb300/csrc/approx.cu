// Batched application of the approximate GFT built in approx.cpp: layers of
// 2x2 units (Haar units, then Jacobi rotations), then the output permutation.
//
// A CTA owns a tile of TS signals, kept NODE-major in shared memory
// (T[node][signal], row stride TSP = TS + 4: rows stay 16-byte aligned and
// sit 4 banks apart).  Within a layer the units touch disjoint nodes, so the
// whole CTA works on one layer at a time: thread item (unit, group of four
// signals) reads the two node rows as 16-byte vectors, applies the unit and
// writes them back; a barrier separates layers.  The tile arrives through a
// transposing copy (a warp moves an 8-node x 4-signal block: 32 distinct
// banks) and leaves through the permutation (coefficient j of signal s is
// T[perm[j]][s]) with 16-byte stores.  Persistent grid.
#include <algorithm>

#include "gft_internal.h"

namespace gft {

namespace {

constexpr int kAThreads = 256;
constexpr int kASmemTarget = 100 * 1024;

struct AArgs {
    const int* pairs;
    const float* coef;
    const int* layer_off;
    const int* perm;
    const float* x;
    float* y;
    long long batch;
    int n, ts, tsp, lg_groups, n_layers;
};

__global__ void __launch_bounds__(kAThreads) approx_fwd_kernel(AArgs a) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float* tile = reinterpret_cast<float*>(sm_raw);
    int* s_perm = reinterpret_cast<int*>(tile + (size_t)a.n * a.tsp);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < a.n; j += kAThreads) s_perm[j] = a.perm[j];
    const long long n_tiles = (a.batch + a.ts - 1) / a.ts;
    const int groups = 1 << a.lg_groups;
    for (long long tl = blockIdx.x; tl < n_tiles; tl += gridDim.x) {
        const int rows = (int)min((long long)a.ts, a.batch - tl * a.ts);
        const float* src = a.x + tl * a.ts * (long long)a.n;
        __syncthreads();   // previous tile stored, permutation loaded
        {
            // transposing load: warp block = 8 nodes x 4 signals
            const int jb = (a.n + 7) >> 3, sb = (rows + 3) >> 2;
            const int jl = lane & 7, sl = lane >> 3;
            for (int blk = warp; blk < jb * sb; blk += kAThreads / 32) {
                const int bs = blk / jb;
                const int j = (blk - bs * jb) * 8 + jl, s = bs * 4 + sl;
                if (j < a.n && s < rows) tile[j * a.tsp + s] = __ldg(src + (long long)s * a.n + j);
            }
        }
        __syncthreads();
        for (int l = 0; l < a.n_layers; ++l) {
            const int u0 = __ldg(a.layer_off + l), u1 = __ldg(a.layer_off + l + 1);
            const int items = (u1 - u0) << a.lg_groups;
            for (int it = tid; it < items; it += kAThreads) {
                const int u = u0 + (it >> a.lg_groups);
                const int g = it & (groups - 1);
                const int p = __ldg(a.pairs + 2 * u), q = __ldg(a.pairs + 2 * u + 1);
                const float4 m = __ldg(reinterpret_cast<const float4*>(a.coef) + u);
                float4* rp = reinterpret_cast<float4*>(tile + p * a.tsp) + g;
                float4* rq = reinterpret_cast<float4*>(tile + q * a.tsp) + g;
                const float4 xp = *rp, xq = *rq;
                *rp = make_float4(fmaf(m.x, xp.x, m.y * xq.x), fmaf(m.x, xp.y, m.y * xq.y),
                                  fmaf(m.x, xp.z, m.y * xq.z), fmaf(m.x, xp.w, m.y * xq.w));
                *rq = make_float4(fmaf(m.z, xp.x, m.w * xq.x), fmaf(m.z, xp.y, m.w * xq.y),
                                  fmaf(m.z, xp.z, m.w * xq.z), fmaf(m.z, xp.w, m.w * xq.w));
            }
            __syncthreads();
        }
        float* dst = a.y + tl * a.ts * (long long)a.n;
        const int E = rows * a.n;
        if ((a.n & 3) == 0) {
            const int per_row = a.n >> 2;
            for (int c = tid; c < (E >> 2); c += kAThreads) {
                const int s = c / per_row, j = 4 * (c - s * per_row);
                __stcs(reinterpret_cast<float4*>(dst) + c,
                       make_float4(tile[s_perm[j] * a.tsp + s], tile[s_perm[j + 1] * a.tsp + s],
                                   tile[s_perm[j + 2] * a.tsp + s], tile[s_perm[j + 3] * a.tsp + s]));
            }
        } else {
            for (int e = tid; e < E; e += kAThreads) {
                const int s = e / a.n, j = e - s * a.n;
                __stcs(dst + e, tile[s_perm[j] * a.tsp + s]);
            }
        }
    }
}

}  // namespace

// Tile shape: the largest TS in {128, 64, 32, 16, 8, 4} whose tile (n rows of
// TS + 4 floats) fits the shared-memory target.
void approx_upload(gft_approx_s& a) {
    const int n = a.n;
    int ts = 128;
    while (ts > 4 && (size_t)n * (ts + 4) * sizeof(float) > (size_t)kASmemTarget) ts >>= 1;
    a.ts = ts;
    a.tsp = ts + 4;
    a.smem = (size_t)n * a.tsp * sizeof(float) + sizeof(int) * (size_t)n;
    if (a.smem > 232448) fail(GFT_ERR_UNSUPPORTED, "graph too large for the approximate-GFT kernel");
    const size_t units = a.pairs.size() / 2;
    std::vector<float> cf(a.coef.begin(), a.coef.end());
    GFT_CUDA(cudaGetDevice(&a.device));
    GFT_CUDA(cudaMalloc(&a.d_pairs, sizeof(int) * std::max<size_t>(2, a.pairs.size())));
    GFT_CUDA(cudaMalloc(&a.d_coef, sizeof(float) * std::max<size_t>(4, cf.size())));
    GFT_CUDA(cudaMalloc(&a.d_layer_off, sizeof(int) * a.layer_off.size()));
    GFT_CUDA(cudaMalloc(&a.d_perm, sizeof(int) * n));
    if (units) {
        GFT_CUDA(cudaMemcpy(a.d_pairs, a.pairs.data(), sizeof(int) * a.pairs.size(), cudaMemcpyHostToDevice));
        GFT_CUDA(cudaMemcpy(a.d_coef, cf.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice));
    }
    GFT_CUDA(cudaMemcpy(a.d_layer_off, a.layer_off.data(), sizeof(int) * a.layer_off.size(), cudaMemcpyHostToDevice));
    GFT_CUDA(cudaMemcpy(a.d_perm, a.perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    a.has_device = true;
}

void approx_free(gft_approx_s& a) {
    if (a.d_pairs) cudaFree(a.d_pairs);
    if (a.d_coef) cudaFree(a.d_coef);
    if (a.d_layer_off) cudaFree(a.d_layer_off);
    if (a.d_perm) cudaFree(a.d_perm);
    a.d_pairs = nullptr;
    a.d_coef = nullptr;
    a.d_layer_off = nullptr;
    a.d_perm = nullptr;
    a.has_device = false;
}

void launch_approx(const gft_approx_s& a, const float* x, float* y, int64_t batch, cudaStream_t st) {
    if (batch <= 0) return;
    AArgs k{};
    k.pairs = a.d_pairs;
    k.coef = a.d_coef;
    k.layer_off = a.d_layer_off;
    k.perm = a.d_perm;
    k.x = x;
    k.y = y;
    k.batch = batch;
    k.n = a.n;
    k.ts = a.ts;
    k.tsp = a.tsp;
    int lg = 0;
    while ((1 << lg) < a.ts / 4) ++lg;
    k.lg_groups = lg;
    k.n_layers = (int)a.layer_off.size() - 1;
    GFT_CUDA(cudaFuncSetAttribute(approx_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem));
    int per_sm = 0;
    GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, approx_fwd_kernel, kAThreads, a.smem));
    if (per_sm < 1) fail(GFT_ERR_UNSUPPORTED, "approximate-GFT kernel does not fit on an SM");
    const long long n_tiles = (batch + a.ts - 1) / a.ts;
    const long long grid = std::min<long long>(n_tiles, (long long)per_sm * sm_count());
    approx_fwd_kernel<<<(unsigned)grid, kAThreads, a.smem, st>>>(k);
    GFT_CUDA(cudaGetLastError());
}

}  // namespace gft

gft_approx_s::~gft_approx_s() { gft::approx_free(*this); }

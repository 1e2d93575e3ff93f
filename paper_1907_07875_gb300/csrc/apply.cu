// CUDA-core fast-GFT transform kernels (FP32 and FP64).
//
// Forward, per signal x (Sec. IV-C, Eq. 13 applied stage by stage):
//   1. every Haar unit (x_i, x_j) -> (x_i + x_j, x_i - x_j), stage by stage
//      (Sec. III: the 1/sqrt(2) of each unit is folded into the leaf matrices);
//   2. every leaf block k: y_k = M_k^T x[I_k] with M_k = diag(2^(-e/2)) U_k;
//   3. coefficients written at their output positions (ascending eigenvalue).
// Inverse: the leaf products with M_k^T, then the stages in reverse order
// (B_phi is its own inverse, Sec. III).
//
// Layout and schedule (GB300):
//   * A CTA owns a tile of TS consecutive signals.  The tile is copied from
//     HBM into shared memory with cp.async (16-byte copies when n is odd,
//     4/8-byte copies otherwise) while the previous tile is being computed
//     (double buffering), so every SM keeps tens of KB of loads in flight.
//   * Shared tiles are row-major with an ODD row stride np (n, or n + 1):
//     thread t works on signal t, so consecutive lanes touch consecutive
//     banks and the per-signal phases are free of bank conflicts.
//   * Each thread owns RS signals of the tile for the whole computation, so
//     the stages and the leaf products need no barrier between them.
//   * Leaf products run IN PLACE: a leaf's inputs are gathered into
//     registers (width bucketed to 4..64 at compile time), and its outputs
//     overwrite those same slots.  The matrix is read from shared memory as
//     4-wide vectors broadcast to the warp; each vector feeds 4*RS FMAs.
//     No separate output tile is needed, which keeps more warps resident.
//   * The output permutation (ascending eigenvalue) is folded into the
//     store: coefficient j of a signal is read from slot src[j] and written
//     with coalesced 16-byte streaming stores.  The inverse applies the same
//     permutation while loading.  Persistent grid: one wave of CTAs loops
//     over tiles.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstdio>

#include "apply_core.cuh"

namespace gft {

namespace {

constexpr int kSmemLimit = 232448;  // 227 KB opt-in per CTA

}  // namespace
using namespace core;
namespace {

template <class T, int RS, int THREADS>
__global__ void __launch_bounds__(THREADS) gft_apply_kernel(KArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [this direction's matrices][program ints, padded to 16 B][nbuf tiles]
    T* mats = reinterpret_cast<T*>(smem_raw);
    int* ints = reinterpret_cast<int*>(smem_raw + sizeof(T) * a.mats_smem);
    const int ints_pad = (a.ints_count + 3) & ~3;
    T* tiles = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(ints) + sizeof(int) * ints_pad);
    const int tile_elems = a.ts * a.np;
    T* buf0 = tiles;
    T* buf1 = tiles + (a.nbuf == 2 ? tile_elems : 0);
    const int tid = threadIdx.x;
    const long long n_tiles = (a.batch + a.ts - 1) / a.ts;
    long long tile = blockIdx.x;

    // program tables first (the inverse load scatters through src)
    for (int i = tid; i < a.ints_count; i += THREADS) ints[i] = a.ints[i];
    __syncthreads();
    const int* src_slot = ints + a.off_src;
    if (tile < n_tiles) issue_tile_load<T, THREADS>(a, src_slot, buf0, tile);
    cp_async_commit();
    {
        const T* gm = reinterpret_cast<const T*>(a.mats);
        const int* desc = ints + a.off_desc;
        for (int k = 0; k < a.n_leaves; ++k) {
            const int bk = desc[kLeafDesc * k + 1];
            const T* src = gm + desc[kLeafDesc * k + 3] + (a.inverse ? bk * bk : 0);
            T* dst = mats + desc[kLeafDesc * k + 4];
            for (int e = tid; e < bk * bk; e += THREADS) dst[e] = src[e];
        }
    }
    int cur = 0;
    for (; tile < n_tiles; tile += gridDim.x) {
        T* buf = cur ? buf1 : buf0;
        const long long nxt = tile + gridDim.x;
        if (a.nbuf == 2) {
            // the other buffer was released by the barrier that ended the
            // previous iteration
            if (nxt < n_tiles) issue_tile_load<T, THREADS>(a, src_slot, cur ? buf0 : buf1, nxt);
            cp_async_commit();
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        __syncthreads();   // tile landed for every thread
        compute_tile<T, RS, THREADS>(a, ints, mats, buf);
        __syncthreads();   // every row computed
        store_tile<T, THREADS>(a, src_slot, buf, tile);
        __syncthreads();   // buffer free for the next load
        if (a.nbuf == 2) {
            cur ^= 1;
        } else {
            if (nxt < n_tiles) issue_tile_load<T, THREADS>(a, src_slot, buf0, nxt);
            cp_async_commit();
        }
    }
    cp_async_wait0();
}

using KFn = void (*)(KArgs);

template <class T>
KFn pick_kernel(int rs, int threads) {
#define GFT_CASE(R, TH) \
    if (rs == R && threads == TH) return gft_apply_kernel<T, R, TH>;
    GFT_CASE(1, 64) GFT_CASE(1, 128) GFT_CASE(1, 256)
    GFT_CASE(2, 64) GFT_CASE(2, 128) GFT_CASE(2, 256)
    GFT_CASE(4, 64) GFT_CASE(4, 128)
#undef GFT_CASE
    return nullptr;
}

struct Cfg {
    int rs, threads, nbuf;
};

int rs_limit(int max_bucket) { return max_bucket <= 16 ? 4 : (max_bucket <= 32 ? 2 : 1); }

template <class T>
size_t smem_bytes(const ApplyArgs& A, const Cfg& c) {
    const size_t fixed = sizeof(T) * (size_t)A.mats_smem + sizeof(int) * (size_t)((A.ints_count + 3) & ~3);
    return fixed + (size_t)c.nbuf * c.rs * c.threads * (A.n | 1) * sizeof(T);
}

// Configuration: an explicit GFT_APPLY_CFG="rs,threads,nbuf" (tuning), else
// the first of a fixed preference list that fits in shared memory.
template <class T>
Cfg choose_cfg(const ApplyArgs& A) {
    const int rmax = rs_limit(A.max_bucket);
    if (const char* e = std::getenv("GFT_APPLY_CFG")) {
        Cfg c{0, 0, 0};
        if (std::sscanf(e, "%d,%d,%d", &c.rs, &c.threads, &c.nbuf) == 3 && c.rs <= rmax &&
            (c.nbuf == 1 || c.nbuf == 2) && pick_kernel<T>(c.rs, c.threads) &&
            smem_bytes<T>(A, c) <= (size_t)kSmemLimit)
            return c;
    }
    const Cfg pref[] = {{2, 128, 2}, {1, 256, 2}, {2, 64, 2}, {1, 128, 2}, {1, 64, 2},
                        {2, 128, 1}, {1, 128, 1}, {1, 64, 1}};
    for (const Cfg& c : pref) {
        if (c.rs > rmax) continue;
        if (sizeof(T) == 8 && c.threads == 256) continue;
        if (smem_bytes<T>(A, c) <= (size_t)kSmemLimit) return c;
    }
    fail(GFT_ERR_UNSUPPORTED, "graph too large for the CUDA-core transform kernel (n=" + std::to_string(A.n) + ")");
}

template <class T>
void launch_apply(const ApplyArgs& A, const T* x, T* y, int64_t batch, bool inverse, cudaStream_t st) {
    if (batch <= 0) return;
    if (A.max_bucket == 0)
        fail(GFT_ERR_UNSUPPORTED, "a leaf has more than 64 nodes; the CUDA-core kernel handles leaves up to 64");
    const Cfg c = choose_cfg<T>(A);
    KArgs k{};
    k.ints = A.ints;
    k.mats = A.mats;
    k.x = x;
    k.y = y;
    k.batch = batch;
    k.n = A.n;
    k.np = A.n | 1;
    k.n_pairs = A.n_pairs;
    k.n_pre_pairs = A.n_pre_pairs;
    k.n_leaves = A.n_leaves;
    k.ints_count = A.ints_count;
    k.off_labels = 2 * A.n_pairs + A.n_stages + 1;
    k.off_outpos = k.off_labels + A.n;
    k.off_src = k.off_outpos + A.n;
    k.off_desc = k.off_src + A.n;
    k.mats_smem = A.mats_smem;
    k.ts = c.rs * c.threads;
    k.nbuf = c.nbuf;
    k.inverse = inverse ? 1 : 0;
    k.inv_n = 1.0f / (float)A.n;
    const size_t smem = smem_bytes<T>(A, c);
    KFn fn = pick_kernel<T>(c.rs, c.threads);
    GFT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, c.threads, smem));
    if (per_sm < 1) fail(GFT_ERR_UNSUPPORTED, "transform kernel does not fit on an SM");
    const long long n_tiles = (batch + k.ts - 1) / k.ts;
    const long long grid = std::min<long long>(n_tiles, (long long)per_sm * sm_count());
    fn<<<(unsigned)grid, c.threads, smem, st>>>(k);
    GFT_CUDA(cudaGetLastError());
}

template <class T>
bool supported(const ApplyArgs& A) {
    if (A.max_bucket == 0) return false;
    const int rmax = rs_limit(A.max_bucket);
    const Cfg pref[] = {{2, 128, 2}, {1, 256, 2}, {2, 64, 2}, {1, 128, 2}, {1, 64, 2},
                        {2, 128, 1}, {1, 128, 1}, {1, 64, 1}};
    for (const Cfg& c : pref) {
        if (c.rs > rmax) continue;
        if (sizeof(T) == 8 && c.threads == 256) continue;
        if (smem_bytes<T>(A, c) <= (size_t)kSmemLimit) return true;
    }
    return false;
}

}  // namespace

bool apply_supported(const ApplyArgs& a, bool f64) { return f64 ? supported<double>(a) : supported<float>(a); }

// SM count of the current device, looked up once per device ordinal
int sm_count() {
    constexpr int kMaxDev = 64;
    static int cached[kMaxDev] = {};
    int dev = 0;
    GFT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) {
        int c = 0;
        GFT_CUDA(cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev));
        return c;
    }
    if (!cached[dev]) {
        int c = 0;
        GFT_CUDA(cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev));
        cached[dev] = c;
    }
    return cached[dev];
}

void launch_apply_f32(const ApplyArgs& a, const float* x, float* y, int64_t batch, bool inverse,
                      cudaStream_t stream) {
    launch_apply<float>(a, x, y, batch, inverse, stream);
}

void launch_apply_f64(const ApplyArgs& a, const double* x, double* y, int64_t batch, bool inverse,
                      cudaStream_t stream) {
    launch_apply<double>(a, x, y, batch, inverse, stream);
}

}  // namespace gft

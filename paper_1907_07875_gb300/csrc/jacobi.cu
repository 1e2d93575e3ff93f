// Batched FP64 Jacobi eigensolver for the leaf Laplacians of a plan.
//
// Every basis U_k of a leaf block is the eigenvector matrix of that block's
// Laplacian (Sec. II-B; the blocks come from Thm. 3 / Eq. 17).  One CTA
// diagonalises one leaf with the parallel-ordering cyclic Jacobi method:
// each sweep runs m-1 rounds of the round-robin tournament, and a round
// rotates m/2 disjoint pairs (p, q) at once, each rotation chosen from the
// 2x2 symmetric Schur decomposition of (a_pp, a_pq, a_qq) so that a_pq
// becomes zero; A <- J^T A J and V <- V J.  Sweeps stop when off(A) <=
// 1e-15 ||A||_F, or fail after 100.
//
// Small leaves keep A and V in shared memory (odd leading dimension, so
// column accesses do not share banks); large leaves work in a global
// scratch copy.  Plan build only: nothing here is on the transform path.
#include <algorithm>
#include <cmath>
#include <memory>
#include <numeric>
#include <vector>

#include "gft_internal.h"

namespace gft {

namespace {

constexpr int kMaxSweeps = 100;
constexpr double kTol = 1e-15;
constexpr int kSmemMaxM = 110;   // 2 * 111 * 111 * 8 bytes fits in 227 KB

struct JacobiJob {
    int m;
    int ld;            // leading dimension of A and V
    long long off;     // offset into A / V buffers (doubles)
};

__device__ __forceinline__ int rr_index(int pos, int round, int me) {
    // circle method: position 0 fixed, the others rotate by one per round
    return pos == 0 ? 0 : ((pos - 1 + round) % (me - 1)) + 1;
}

__device__ __forceinline__ void schur2(double app, double aqq, double apq, double& c, double& s) {
    if (apq == 0.0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    const double tau = (aqq - app) / (2.0 * apq);
    // smaller root of t^2 + 2 tau t - 1 = 0
    const double t = (tau >= 0.0) ? 1.0 / (tau + hypot(1.0, tau)) : -1.0 / (-tau + hypot(1.0, tau));
    c = 1.0 / sqrt(1.0 + t * t);
    s = t * c;
}

// Block-wide sum of a double (blockDim.x a multiple of 32, <= 1024).
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) r += red[i];
    __syncthreads();
    return r;
}

// A, V point at this leaf's storage (shared or global), leading dim ld.
__device__ void jacobi_core(double* A, double* V, int m, int ld, double* cs, int* pq, double* red,
                            int* sweeps_out, int* ok_out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int me = m + (m & 1);
    const int half = me / 2;
    double fro2 = 0.0;
    for (int e = tid; e < m * m; e += nt) {
        const double a = A[(e / m) * ld + (e % m)];
        fro2 += a * a;
    }
    fro2 = block_sum(fro2, red);
    int sweep = 0;
    bool done = false;
    while (true) {
        double off2 = 0.0;
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, j = e % m;
            if (i != j) {
                const double a = A[i * ld + j];
                off2 += a * a;
            }
        }
        off2 = block_sum(off2, red);
        if (off2 <= kTol * kTol * fro2) {
            done = true;
            break;
        }
        if (sweep == kMaxSweeps) break;
        ++sweep;
        for (int round = 0; round < me - 1; ++round) {
            for (int k = tid; k < half; k += nt) {
                int p = rr_index(k, round, me), q = rr_index(me - 1 - k, round, me);
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                double c = 1.0, s = 0.0;
                int act = 0;
                if (q < m) {
                    const double apq = A[p * ld + q];
                    if (apq != 0.0) {
                        schur2(A[p * ld + p], A[q * ld + q], apq, c, s);
                        act = 1;
                    }
                }
                cs[2 * k] = c;
                cs[2 * k + 1] = s;
                pq[2 * k] = act ? p : -1;
                pq[2 * k + 1] = q;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = tid; e < half * m; e += nt) {
                const int k = e / m, i = e % m;
                const int p = pq[2 * k];
                if (p < 0) continue;
                const int q = pq[2 * k + 1];
                const double c = cs[2 * k], s = cs[2 * k + 1];
                const double ap = A[i * ld + p], aq = A[i * ld + q];
                A[i * ld + p] = c * ap - s * aq;
                A[i * ld + q] = s * ap + c * aq;
                const double vp = V[i * ld + p], vq = V[i * ld + q];
                V[i * ld + p] = c * vp - s * vq;
                V[i * ld + q] = s * vp + c * vq;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < half * m; e += nt) {
                const int k = e / m, j = e % m;
                const int p = pq[2 * k];
                if (p < 0) continue;
                const int q = pq[2 * k + 1];
                const double c = cs[2 * k], s = cs[2 * k + 1];
                const double ap = A[p * ld + j], aq = A[q * ld + j];
                A[p * ld + j] = c * ap - s * aq;
                A[q * ld + j] = s * ap + c * aq;
            }
            __syncthreads();
            for (int k = tid; k < half; k += nt) {
                const int p = pq[2 * k];
                if (p < 0) continue;
                const int q = pq[2 * k + 1];
                A[p * ld + q] = 0.0;
                A[q * ld + p] = 0.0;
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        *sweeps_out = sweep;
        *ok_out = done ? 1 : 0;
    }
}

__global__ void jacobi_smem_kernel(const JacobiJob* jobs, double* gA, double* gV, int* sweeps, int* ok) {
    extern __shared__ double sm[];
    const JacobiJob jb = jobs[blockIdx.x];
    const int m = jb.m, ld = jb.ld;
    double* A = sm;
    double* V = A + (size_t)m * ld;
    double* cs = V + (size_t)m * ld;         // 2 * half
    double* red = cs + (m + 1);              // 32
    int* pq = (int*)(red + 32);              // 2 * half
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        A[i * ld + j] = gA[jb.off + (long long)i * m + j];
        V[i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    jacobi_core(A, V, m, ld, cs, pq, red, &sweeps[blockIdx.x], &ok[blockIdx.x]);
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        gA[jb.off + (long long)i * m + j] = A[i * ld + j];
        gV[jb.off + (long long)i * m + j] = V[i * ld + j];
    }
}

// Large leaves: A and V live in global scratch (leading dimension m).
__global__ void jacobi_global_kernel(const JacobiJob* jobs, double* gA, double* gV, int* sweeps, int* ok) {
    extern __shared__ double sm[];
    const JacobiJob jb = jobs[blockIdx.x];
    const int m = jb.m;
    double* A = gA + jb.off;
    double* V = gV + jb.off;
    double* cs = sm;
    double* red = cs + (m + 1);
    int* pq = (int*)(red + 32);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) V[e] = ((e / m) == (e % m)) ? 1.0 : 0.0;
    __syncthreads();
    jacobi_core(A, V, m, m, cs, pq, red, &sweeps[blockIdx.x], &ok[blockIdx.x]);
}

template <class T>
struct DevBuf {
    T* p = nullptr;
    DevBuf() = default;
    explicit DevBuf(size_t n) {
        if (n) GFT_CUDA(cudaMalloc(&p, n * sizeof(T)));
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p) { o.p = nullptr; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            if (p) cudaFree(p);
            p = o.p;
            o.p = nullptr;
        }
        return *this;
    }
};

}  // namespace

// Every leaf of every plan in one batched solve: 1x1 leaves on the host,
// the others grouped by size (shared-memory kernel for m <= 16, 32, 64,
// 110, so each launch sizes its shared memory to its own largest leaf; the
// global-memory kernel above) -- the large group on its own stream, so it
// overlaps the small ones.
void jacobi_leaf_ptrs(const std::vector<Leaf*>& leaves, cudaStream_t stream) {
    std::vector<std::vector<int>> groups(5);
    const int lim[4] = {16, 32, 64, kSmemMaxM};
    for (size_t k = 0; k < leaves.size(); ++k) {
        Leaf& lf = *leaves[k];
        const int m = lf.m();
        if (m == 1) {
            lf.lam = {lf.L[0]};
            lf.V = {1.0};
            lf.sweeps = 0;
            continue;
        }
        int g = 4;
        for (int b = 0; b < 4; ++b)
            if (m <= lim[b]) {
                g = b;
                break;
            }
        groups[g].push_back((int)k);
    }
    struct Run {
        std::vector<int> ids;
        std::vector<JacobiJob> jobs;
        std::vector<double> hA, hV;
        std::vector<int> hS, hOk;
        DevBuf<double> dA, dV;
        DevBuf<JacobiJob> dJ;
        DevBuf<int> dS, dOk;
    };
    cudaStream_t big = nullptr;
    GFT_CUDA(cudaStreamCreateWithFlags(&big, cudaStreamNonBlocking));
    std::vector<std::unique_ptr<Run>> runs;
    try {
        for (int g = 4; g >= 0; --g) {   // large leaves first: they take longest
            if (groups[g].empty()) continue;
            const bool in_smem = g < 4;
            cudaStream_t st = in_smem ? stream : big;
            std::unique_ptr<Run> R(new Run);
            R->ids = groups[g];
            long long total = 0;
            int maxm = 0;
            for (int k : R->ids) {
                const int m = leaves[k]->m();
                R->jobs.push_back({m, in_smem ? (m | 1) : m, total});
                total += (long long)m * m;
                maxm = std::max(maxm, m);
            }
            R->hA.resize((size_t)total);
            for (size_t j = 0; j < R->ids.size(); ++j) {
                const Leaf& lf = *leaves[R->ids[j]];
                std::copy(lf.L.begin(), lf.L.end(), R->hA.begin() + R->jobs[j].off);
            }
            const int B = (int)R->ids.size();
            R->dA = DevBuf<double>(total);
            R->dV = DevBuf<double>(total);
            R->dJ = DevBuf<JacobiJob>(B);
            R->dS = DevBuf<int>(B);
            R->dOk = DevBuf<int>(B);
            GFT_CUDA(cudaMemcpyAsync(R->dA.p, R->hA.data(), sizeof(double) * total, cudaMemcpyHostToDevice, st));
            GFT_CUDA(cudaMemcpyAsync(R->dJ.p, R->jobs.data(), sizeof(JacobiJob) * B, cudaMemcpyHostToDevice, st));
            const size_t aux = sizeof(double) * ((maxm + 1) + 32) + sizeof(int) * (maxm + 1);
            if (in_smem) {
                const int ld = maxm | 1;
                const size_t smem = sizeof(double) * 2 * (size_t)maxm * ld + aux;
                GFT_CUDA(cudaFuncSetAttribute(jacobi_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                const int threads = maxm <= 32 ? 128 : 256;
                jacobi_smem_kernel<<<B, threads, smem, st>>>(R->dJ.p, R->dA.p, R->dV.p, R->dS.p, R->dOk.p);
            } else {
                jacobi_global_kernel<<<B, 1024, aux, st>>>(R->dJ.p, R->dA.p, R->dV.p, R->dS.p, R->dOk.p);
            }
            GFT_CUDA(cudaGetLastError());
            R->hV.resize((size_t)total);
            R->hS.resize(B);
            R->hOk.resize(B);
            GFT_CUDA(cudaMemcpyAsync(R->hA.data(), R->dA.p, sizeof(double) * total, cudaMemcpyDeviceToHost, st));
            GFT_CUDA(cudaMemcpyAsync(R->hV.data(), R->dV.p, sizeof(double) * total, cudaMemcpyDeviceToHost, st));
            GFT_CUDA(cudaMemcpyAsync(R->hS.data(), R->dS.p, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
            GFT_CUDA(cudaMemcpyAsync(R->hOk.data(), R->dOk.p, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
            runs.push_back(std::move(R));
        }
        GFT_CUDA(cudaStreamSynchronize(stream));
        GFT_CUDA(cudaStreamSynchronize(big));
    } catch (...) {
        cudaStreamSynchronize(stream);
        cudaStreamSynchronize(big);
        cudaStreamDestroy(big);
        throw;
    }
    GFT_CUDA(cudaStreamDestroy(big));
    for (auto& R : runs) {
        for (size_t j = 0; j < R->ids.size(); ++j) {
            Leaf& lf = *leaves[R->ids[j]];
            const int m = lf.m();
            if (!R->hOk[j])
                fail(GFT_ERR_NO_CONVERGENCE, "Jacobi did not converge for leaf '" + lf.tag + "' (m=" +
                                                 std::to_string(m) + ")");
            const double* A = R->hA.data() + R->jobs[j].off;
            const double* V = R->hV.data() + R->jobs[j].off;
            std::vector<int> ord(m);
            std::iota(ord.begin(), ord.end(), 0);
            std::stable_sort(ord.begin(), ord.end(),
                             [&](int a, int b) { return A[(size_t)a * m + a] < A[(size_t)b * m + b]; });
            lf.lam.resize(m);
            lf.V.assign((size_t)m * m, 0.0);
            for (int c = 0; c < m; ++c) {
                lf.lam[c] = A[(size_t)ord[c] * m + ord[c]];
                for (int r = 0; r < m; ++r) lf.V[(size_t)r * m + c] = V[(size_t)r * m + ord[c]];
            }
            lf.sweeps = R->hS[j];
        }
    }
}

void jacobi_leaves(std::vector<Leaf>& leaves, cudaStream_t stream) {
    std::vector<Leaf*> ptrs;
    for (auto& lf : leaves) ptrs.push_back(&lf);
    jacobi_leaf_ptrs(ptrs, stream);
}

}  // namespace gft

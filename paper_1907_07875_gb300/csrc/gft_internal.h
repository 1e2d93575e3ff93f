// Internal declarations of the GB300 fast-GFT library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "gft.h"

namespace gft {

// ---------------------------------------------------------------------------
// errors: internal code throws GftError; the extern "C" layer converts it to
// a status code and records the message for gft_last_error().
// ---------------------------------------------------------------------------
struct GftError {
    gft_status code;
    std::string msg;
};
[[noreturn]] void fail(gft_status code, const std::string& msg);
void set_last_error(const std::string& msg);
void cuda_check(cudaError_t e, const char* what);
#define GFT_CUDA(call) ::gft::cuda_check((call), #call)

// device-side error word values (written by kernels, read by the host)
enum DevErr : int { kDevOk = 0, kDevTimeout = GFT_ERR_TIMEOUT, kDevBadShape = GFT_ERR_INVALID_ARG };

// ---------------------------------------------------------------------------
// plan (host side)
// ---------------------------------------------------------------------------
struct Leaf {
    std::vector<int> labels;   // original labels in leaf order
    std::vector<double> L;     // m*m leaf Laplacian, row-major
    std::vector<int> exps;     // per node: Haar stages its lineage took part in
    std::vector<int> cexps;    // per column: output-side (right) Haar units it feeds (empty = none)
    std::string tag;           // "+"/"-" path (plus ".c" for a component)
    // after eigendecomposition
    std::vector<double> lam;   // ascending
    std::vector<double> V;     // m*m row-major: V[r*m + c] = entry r of eigenvector c
    int sweeps = 0;
    int m() const { return (int)labels.size(); }
    // Folded matrix entry M[r][c] = 2^(-e_r/2) V[r][c] 2^(-f_c/2): the
    // 1/sqrt2 of every Haar unit the row's input went through (left stages)
    // or the column's output goes through (right stage).
    double fold(int r, int c) const {
        const int e = exps[r] + (cexps.empty() ? 0 : cexps[c]);
        return std::pow(2.0, -0.5 * e) * V[(size_t)r * m() + c];
    }
};

// Bucketed leaf width used by the CUDA-core kernels (registers are sized at
// compile time): 4, 8, 16, 24, 32, 48, 64.  0 = too large for CUDA cores.
int leaf_bucket(int m);
constexpr int kMaxCoreLeaf = 64;

// Everything a CUDA-core transform kernel needs, in one device allocation.
//   ints:  [pairs 2P][stage_off S+1][labels n][out_pos n][src n][leaf desc 5L]
//   pairs of the first n_pre_stages stages act on the input (before the
//   leaf products), the rest on the leaf outputs (right Haar units, slot
//   pairs): P = n_pre_pairs + right pairs, S = n_pre_stages + (0 or 1)
//   src[j] = tile slot (node label) that holds coefficient j after the
//          in-place leaf products
//   leaf desc = {m, bucket, off (into labels/out_pos), off_u (into mats),
//                off_s (into the per-direction matrices held in smem)}
//   mats:  per leaf, the forward matrix M_f (bucket x bucket, row-major,
//          M_f[r][c] = 2^(-e_r/2) V[r][c], zero padded) followed by the
//          inverse matrix M_i = M_f^T (same padding)
struct DevProgram {
    int n = 0, n_stages = 0, n_leaves = 0, n_pairs = 0;
    int n_pre_stages = 0, n_pre_pairs = 0;
    int max_bucket = 0;
    int ints_count = 0;      // int32 entries
    int mats_count = 0;      // scalars per precision (both directions)
    int mats_smem = 0;       // scalars of one direction's matrices
    int* d_ints = nullptr;
    float* d_mats32 = nullptr;
    double* d_mats64 = nullptr;
    int* d_err = nullptr;    // device error word
    // node-major batch kernel's program image (CUDA-core plans only):
    // [ints, padded to 4][(leaf << 16 | first output) per group of four
    // outputs, padded to 4]
    int* d_nm = nullptr;
    int nm_words = 0, nm_cg_off = 0, nm_n_cg = 0;
};

// tcn.cu: tensor-core leaf products with the signals on the MMA's N axis,
// for mixed batches of graphs with few signals each (leaves up to 512)
bool tcn_eligible(const gft_plan_s& p);
void tcn_free(gft_plan_s& p);
void* tcn_batch_create(const std::vector<gft_plan_s*>& plans, const std::vector<int64_t>& batches, uint32_t precision);
void tcn_batch_upload(void* tb, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st);
void tcn_batch_launch(void* tb, cudaStream_t st);
void tcn_batch_free(void* tb);
int tcn_batch_launches(void* tb);

}  // namespace gft

struct gft_plan_s {
    int n = 0;
    uint32_t flags = 0;
    int n_stages = 0;
    std::vector<double> L;                                  // n*n
    std::vector<std::vector<std::pair<int, int>>> stages;   // (X label, partner)
    std::vector<gft::Leaf> leaves;
    // right Haar stage (bipartite plans, Sec. III-A): leaves[0] = E on the
    // larger part, leaves[1] = F on the smaller; column c < p of E and of F
    // form one unit, its sum in E's slot, its difference in F's slot
    bool right = false;
    double alpha = 0.0;                                     // L[S,S] = alpha I on both parts
    std::vector<std::pair<int, int>> rpairs;                // (slot of E column c, slot of F column c)
    bool has_device = false;
    std::vector<int> out_pos;      // n, leaf-concatenated order -> coefficient
    std::vector<double> lam_out;   // n, coefficient order
    gft::DevProgram dev;
    cudaStream_t last_stream = nullptr;
    int device = 0;
    // host-batch staging (gft_plan_forward_host): one in/out buffer pair per stream
    static constexpr int kHostStreams = 3;
    float* d_stage[kHostStreams] = {};
    float* d_stage_out[kHostStreams] = {};
    size_t stage_elems = 0;
    cudaStream_t host_streams[kHostStreams] = {};   // upload, compute, download
    cudaEvent_t ev_up[kHostStreams] = {}, ev_k[kHostStreams] = {}, ev_down[kHostStreams] = {};
    // tensor-core data (built lazily)
    void* tc = nullptr;
    // tensor-core data of the few-signals batch kernel (tcn.cu; built lazily)
    void* tcn = nullptr;
    // plan-specialised kernels (jit.cpp)
    void* jit = nullptr;
    // wide-leaf CUDA-core kernel data (wide.cu)
    void* wide = nullptr;
    ~gft_plan_s();
};

// Approximate GFT (Sec. VI-B): Haar stages, then greedy layers of Jacobi
// rotations per leaf, then the output permutation (approx.cpp / approx.cu).
struct gft_approx_s {
    int n = 0, n_stages = 0, n_haar_layers = 0;
    std::vector<int> layer_off;     // layers + 1: units of layer l are [layer_off[l], layer_off[l+1])
    std::vector<int> pairs;         // 2 per unit (p, q)
    std::vector<double> coef;       // 4 per unit: (x_p, x_q) <- (m00 x_p + m01 x_q, m10 x_p + m11 x_q)
    std::vector<int> perm;          // coefficient j is read from node perm[j]
    std::vector<double> lam;        // approximate eigenvalues, output order
    bool has_device = false;
    int device = 0;
    int ts = 0, tsp = 0;            // signals per tile, node-row stride of the shared tile
    size_t smem = 0;
    int* d_pairs = nullptr;
    float* d_coef = nullptr;
    int* d_layer_off = nullptr;
    int* d_perm = nullptr;
    cudaStream_t last_stream = nullptr;
    ~gft_approx_s();
};

namespace gft {

// approx.cpp / approx.cu
void approx_build(gft_approx_s& a, const double* L, int n_stages, const int32_t* phi, int n_layers, uint32_t flags);
void approx_upload(gft_approx_s& a);
void approx_free(gft_approx_s& a);
void launch_approx(const gft_approx_s& a, const float* x, float* y, int64_t batch, cudaStream_t st);

// plan.cpp
void analyze(gft_plan_s& p, const double* L, int n_stages, const int32_t* phi);
// output index of every entry (eigenvalue, leaf, index in leaf): ascending
// eigenvalue; values within 1e-9 max(1, |lam|max) of a neighbour form a
// cluster ordered by (leaf, index)
std::vector<int> output_positions(const std::vector<double>& lam, const std::vector<int>& leaf,
                                  const std::vector<int>& local);
// bipartite plan with a right Haar stage: validation, parts, and the
// coupling-block matrix whose eigendecomposition gives E and F
void analyze_bipartite(gft_plan_s& p, const double* L, const int32_t* side, Leaf& coupling);
void finish_bipartite(gft_plan_s& p, const Leaf& coupling);   // E, F, sigma from the solved coupling leaf
void finalize_host(gft_plan_s& p);           // ordering, signs
void upload_plan(gft_plan_s& p);             // device program
void compute_basis(const gft_plan_s& p, double* U);
void free_device(gft_plan_s& p);

// jacobi.cu: eigendecompose every leaf on the current device (FP64).
void jacobi_leaves(std::vector<Leaf>& leaves, cudaStream_t stream);
void jacobi_leaf_ptrs(const std::vector<Leaf*>& leaves, cudaStream_t stream);   // leaves of many plans

// apply.cu
struct ApplyArgs {
    const int* ints;
    const void* mats;       // float* or double*
    int n, n_stages, n_leaves, n_pairs, max_bucket;
    int n_pre_pairs;        // pairs applied before the leaf products
    int ints_count, mats_count, mats_smem;
    int* err;
};
constexpr int kLeafDesc = 5;
void launch_apply_f32(const ApplyArgs& a, const float* x, float* y, int64_t batch, bool inverse,
                      cudaStream_t stream);
void launch_apply_f64(const ApplyArgs& a, const double* x, double* y, int64_t batch, bool inverse,
                      cudaStream_t stream);
ApplyArgs apply_args(const gft_plan_s& p, bool f64);
bool apply_supported(const ApplyArgs& a, bool f64);   // the table-driven kernel fits this plan
int sm_count();

// jit.cpp: plan-specialised kernels
bool jit_eligible(const gft_plan_s& p);
void jit_build(gft_plan_s& p);
void jit_free(gft_plan_s& p);
bool jit_launch(gft_plan_s& p, bool f64, const void* x, void* y, int64_t batch, bool inverse, cudaStream_t st);
void jit_info(const gft_plan_s& p, int* jit, int* tile, int* threads);
bool jit_launch_plain(gft_plan_s& p, const float* x, float* y, int64_t batch, cudaStream_t st);
std::string jit_source(const gft_plan_s& p, bool f64);
// plan-specialised group of a mixed batch (small plans shared by many entries)
bool jit_group_eligible(const gft_plan_s& p);
void* jit_group_create(const std::vector<gft_plan_s*>& plans, const std::vector<int64_t>& batches);
void jit_group_upload(void* g, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st);
void jit_group_launch(void* g, cudaStream_t st);
void jit_group_free(void* g);
int jit_group_launches(void* g);
int jit_group_tile(void* g, int entry);

// search.cpp: involution search (Sec. V-F)
int find_involution(int n, const double* L, const int* classes, long long max_steps, double scale, int* phi);
int search_stages(int n, const double* L, int max_stages, long long max_steps, std::vector<int>& phis);

// wide.cu: CUDA-core kernel for leaves wider than 32 nodes (up to 512)
bool wide_eligible(const gft_plan_s& p);
void wide_build(gft_plan_s& p);
void wide_free(gft_plan_s& p);
bool wide_ready(const gft_plan_s& p, bool f64);
void launch_wide_f32(gft_plan_s& p, const float* x, float* y, int64_t batch, bool inverse, cudaStream_t st);
void launch_wide_f64(gft_plan_s& p, const double* x, double* y, int64_t batch, bool inverse, cudaStream_t st);
bool wide_configured(const gft_plan_s& p);    // an FP32 wide-leaf configuration exists
// mixed batches of wide-leaf plans: one persistent FP32 forward launch
void* wide_batch_create(const std::vector<gft_plan_s*>& plans, const std::vector<int64_t>& batches);
void wide_batch_upload(void* wb, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st);
void wide_batch_launch(void* wb, cudaStream_t st);
void wide_batch_free(void* wb);
int wide_batch_launches(void* wb);

// tc.cu: leaf products on tcgen05 tensor cores (split precision)
bool tc_eligible(const gft_plan_s& p);
void tc_build(gft_plan_s& p);
void tc_free(gft_plan_s& p);
// Device scratch of the tensor-core path: a plan holds one for its own
// transforms; a mixed batch holds one per tensor-core plan so that its
// captured graph never sees the plan's scratch move.
struct TcScratch {
    unsigned char* d_aimg = nullptr;   // A images, [tiles][items] x 32 KB
    float* d_scale = nullptr;          // per-signal FP16 scale
    float* d_z = nullptr;              // leaf-ordered output (several TMEM groups)
    size_t rows_cap = 0;
    void release();
    ~TcScratch() { release(); }
};
void tc_reserve(gft_plan_s& p, TcScratch& s, int64_t batch);   // builds the tensor-core data on first use
void launch_tc(gft_plan_s& p, const float* x, float* y, int64_t batch, bool inverse, cudaStream_t st,
               uint32_t precision, TcScratch* scratch = nullptr);
// mixed batches: every tensor-core plan in one pack and one leaf launch per size class
void* tc_batch_create(const std::vector<gft_plan_s*>& plans, const std::vector<int64_t>& batches, uint32_t precision);
void tc_batch_upload(void* tb, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st);
void tc_batch_launch(void* tb, cudaStream_t st);
void tc_batch_free(void* tb);
int tc_batch_launches(void* tb);

// tcn.cu: tensor-core leaf products with the signals on the MMA's N axis,
// for mixed batches of graphs with few signals each (leaves up to 512)
bool tcn_eligible(const gft_plan_s& p);
void tcn_free(gft_plan_s& p);
void* tcn_batch_create(const std::vector<gft_plan_s*>& plans, const std::vector<int64_t>& batches, uint32_t precision);
void tcn_batch_upload(void* tb, const std::vector<const float*>& x, const std::vector<float*>& y, cudaStream_t st);
void tcn_batch_launch(void* tb, cudaStream_t st);
void tcn_batch_free(void* tb);
int tcn_batch_launches(void* tb);

}  // namespace gft

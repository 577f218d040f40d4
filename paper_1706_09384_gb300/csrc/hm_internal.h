// hm_internal.h — internal declarations shared by the libhm CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/hm.h"
#include "green.cuh"

// Thrown inside the library only; every entry point converts it to an hm_status.
struct hm_error {
    hm_status st;
    std::string msg;
};
void hm_set_error(const std::string& msg);
[[noreturn]] void hm_throw(hm_status st, const std::string& msg);
void hm_check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define HM_CUDA(call) hm_check_cuda((call), #call, __FILE__, __LINE__)

// Kernel launch counter (reported by hm_kernel_launches).
extern std::atomic<long long> g_hm_launches;
#define HM_LAUNCHED() g_hm_launches.fetch_add(1, std::memory_order_relaxed)

// Solver and build scratch (scratch.cu): stream-ordered allocations from the
// library's per-device pool, which keeps freed memory for reuse; and small
// pinned host buffers from a process-wide free list.
void* hm_scratch_alloc(size_t bytes, cudaStream_t st);
void hm_scratch_free(void* p, cudaStream_t st);
size_t hm_scratch_cached();  // bytes the current device's pool holds but does not use
void hm_scratch_trim();      // returns every pool's unused memory to its device
void* hm_pinned_take(size_t bytes);
void hm_pinned_give(void* p);
// One page-locked int from that free list, returned when it goes out of scope.
struct PinnedInt {
    int* p;
    PinnedInt() : p((int*)hm_pinned_take(sizeof(int))) { *p = 0; }
    ~PinnedInt() { hm_pinned_give(p); }
    PinnedInt(const PinnedInt&) = delete;
    PinnedInt& operator=(const PinnedInt&) = delete;
};

// Device allocation owned by the handle (freed in hm_free).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    bool pooled = false;            // from the library's pool: freed on `st`, stays reserved
    cudaStream_t st = nullptr;
};
void* hm_dmalloc(std::vector<DevBuf>& owner, size_t bytes, cudaStream_t st, bool zero);
// The same from the library's stream-ordered pool (build workspaces: the ACA
// factors, the staged factors): released on `st` by free_all, the memory
// stays reserved for the next build until hm_release_cached_memory.
void* hm_dmalloc_pooled(std::vector<DevBuf>& owner, size_t bytes, cudaStream_t st);

// ---------------- tree + partition (tree.cu) ----------------
struct TreeResult {
    std::vector<hm_cluster> clusters;   // BFS order, root = 0
    std::vector<int64_t> perm;          // perm[p] = original index at tree position p
    int depth = 0;
};
// pts_p (device, n x 3) is permuted in place into tree order; d_perm receives perm.
TreeResult build_cluster_tree(double* d_pts, int64_t* d_perm, int64_t nc, int64_t leaf,
                              cudaStream_t st);
// Level-synchronous block-cluster-tree traversal (Sec. 2.1) with the box
// admissibility of Sec. 6.1, from the root pair (0, sigma_root): 0 for one
// cloud; for two clouds the targets' tree comes first in cl and sigma_root is
// the sources' root.  Returns blocks (tau, sigma, admissible) in level order.
std::vector<hm_block> build_partition(const std::vector<hm_cluster>& cl, double eta,
                                      cudaStream_t st, int64_t sigma_root = 0);

// ---------------- matvec storage plan (matvec.cu) ----------------
// Storage segments: the leaf clusters, each cut into the fewest contiguous
// point ranges of at most 64 points (a leaf of up to 64 points is one segment).
// One chunk = rows of one segment of a block's row set (dense block, U
// factor) or column set (V factor); column-major with ld = padded rows.
struct Chunk {
    int64_t data;      // element offset (complex) into the arena
    int32_t ld;        // padded row count (even)
    int32_t rows;      // 3 |leaf|
    int32_t ncols;     // dense: 3|sigma|; factors: rank
    int32_t kind;      // 0 dense, 1 U, 2 V
    int64_t vec;       // dense: x offset (tree order DOF); U/V: t offset
    int64_t block;     // block index
    int64_t sigma;     // column cluster of the block
    int64_t leaf_dof;  // first tree-order DOF of the chunk's segment
};

struct MatvecPlan {
    // per segment (row side): list of dense + U chunks; per segment (col side): V chunks
    std::vector<int64_t> row_leaf_begin;   // CSR over segments
    std::vector<int32_t> row_items;        // chunk ids
    std::vector<int64_t> col_leaf_begin;
    std::vector<int32_t> col_items;
    std::vector<Chunk> chunks;
    std::vector<int64_t> leaf_dof_begin;   // first DOF (tree order) of each segment
    std::vector<int32_t> leaf_rows;        // 3 |segment| (<= MAX_LD)
    int64_t arena_elems = 0;               // complex entries in the arena
    int64_t t_elems = 0;                   // entries of the t = V^H x workspace
};

MatvecPlan build_matvec_plan(const std::vector<hm_cluster>& cl, const std::vector<hm_block>& blk,
                             std::vector<int64_t>& t_off);
struct MatvecDev;  // device side of the plan (matvec.cu)
MatvecDev* matvec_dev_create(const MatvecPlan& plan, int storage, std::vector<DevBuf>& owner,
                             cudaStream_t st);
void matvec_dev_destroy(MatvecDev* m);
// Products over the items of the active segments only (segment q = DOFs
// [dof_bounds[q], dof_bounds[q + 1])); all active restores the full lists.
void matvec_select_segments(MatvecDev* m, const std::vector<int64_t>& dof_bounds,
                            const std::vector<int>& act, cudaStream_t st);
// Launch parameters of the one-vector product picked by the autotuner: stages
// of the streamed BF16 kernels (2..4) and, with FP32 storage, the byte size of
// a work item (re-tiles the items).
void matvec_set_params(MatvecDev* m, const MatvecPlan& plan, int s16_nstage, int64_t item_bytes,
                       cudaStream_t st);
// Adds the BF16 copy of the arena (per-chunk FP32 scale); the fast product then
// reads it, the accurate product keeps reading the FP32 arena.
void matvec_make_bf16(MatvecDev* m, const MatvecPlan& plan, std::vector<DevBuf>& owner,
                      cudaStream_t st);
void* matvec_arena(MatvecDev* m);           // float2* (fp32) or bf16 pairs
// y (original order, complex128) = A_H x through the product's CUDA graph;
// xp, yp: tree-order complex64 scratch owned by the caller, fixed per handle.
void matvec_graph(MatvecDev* m, const int64_t* d_perm, const double2* x, float2* xp, float2* yp,
                  double2* y, int64_t nc, cudaStream_t st);
// Captures and instantiates that graph ahead of the first product (no-op once
// it exists), so the build pays for it instead of the caller's first product.
void matvec_graph_prepare(MatvecDev* m, const int64_t* d_perm, float2* xp, float2* yp, int64_t nc);
// Error code left by the streamed product kernels (0 = none; 1 = a wait on a
// copy gave up); reading it synchronises st and clears it.
int matvec_take_error(MatvecDev* m, cudaStream_t st);
// The same in two parts, so the readback shares the caller's synchronisation:
// queue the copy of the code into page-locked `pinned` on st, then, once st has
// synchronised, read it (a set code is cleared on st).
void matvec_queue_error(MatvecDev* m, int* pinned, cudaStream_t st);
int matvec_read_error(MatvecDev* m, const int* pinned, cudaStream_t st);
// Y = A_H X for nrhs right-hand sides (complex128, 3 nc x nrhs column-major,
// original order) on the tensor cores, in blocks of 32; BF16 storage only.
void matvec_multi(MatvecDev* m, const int64_t* d_perm, const double2* x, double2* y, int64_t nc,
                  int32_t nrhs, cudaStream_t st);
// algorithmic bytes of one 32-right-hand-side block product (stored entries + vectors)
int64_t matvec_multi_alg_bytes(const MatvecDev* m, int64_t ndof);
// mean device ms of gather, phase 1, phase 2, scatter of one 32-column block product
void matvec_multi_profile(MatvecDev* m, const int64_t* d_perm, const double2* x, double2* y,
                          int64_t nc, int32_t reps, double ms[4], cudaStream_t st);
// y_p (tree order, float2) = A_H x_p (tree order, float2)
void matvec_tree_order(MatvecDev* m, const float2* xp, float2* yp, int64_t ndof, cudaStream_t st);
// Copies staged column-major blocks / factors (FP32, one pointer per block:
// dense block or U in src_u, V in src_v, leading dimension 3|tau| / 3|sigma|)
// into the chunks of the arena.
void copy_staged_chunks(MatvecDev* m, const MatvecPlan& plan, const std::vector<hm_block>& blk,
                        const std::vector<hm_cluster>& cl, const std::vector<const float2*>& src_u,
                        const std::vector<const float2*>& src_v, cudaStream_t st);
// Gather/scatter between original order (complex128) and tree order (complex64).
void launch_gather_x(const int64_t* d_perm, const double2* x, float2* xp, int64_t nc,
                     cudaStream_t st);
void launch_scatter_y(const int64_t* d_perm, const float2* yp, double2* y, int64_t nc,
                      cudaStream_t st);
// Accurate product (FP32-stored entries, x / t and the sums as double-float
// pairs of FP32 numbers, results in complex128), used for
// the true residual of GMRES restarts.  xp64, yp64: tree-order scratch (3 nc).
void matvec_accurate(MatvecDev* m, const int64_t* d_perm, const double2* x, double2* xp64,
                     double2* yp64, double2* y, int64_t nc, cudaStream_t st);
// The three parts of the product, for per-kernel timing.
void matvec_phase1(MatvecDev* m, const float2* xp, cudaStream_t st);
void matvec_phase2(MatvecDev* m, const float2* xp, float2* yp, int64_t ndof, cudaStream_t st);
// algorithmic bytes: [0] phase 1, [1] phase 2, [2] whole product (given ndof)
void matvec_alg_bytes(const MatvecDev* m, int64_t ndof, int64_t out[3]);
int64_t matvec_stored_bytes(const MatvecDev* m);
int64_t matvec_dense_bytes(const MatvecDev* m);

// ---------------- near field (nearfield.cu) ----------------
// Writes all dense chunks (kind 0) of the plan into the FP32 arena.
void assemble_dense(const GreenParams& gp, const double* d_pts_p, const double* d_nrm_p,
                    const MatvecPlan& plan, const std::vector<hm_block>& blocks,
                    const std::vector<hm_cluster>& cl, MatvecDev* mv, std::vector<DevBuf>& owner,
                    cudaStream_t st);
void launch_green_eval(const GreenParams& gp, const double* x, const double* y,
                       const double* ny, int64_t npairs, double2* out, cudaStream_t st);

// ---------------- ACA + recompression (aca.cu, recompress.cu) ----------------
struct AcaJob {              // one admissible block
    int64_t tau_begin, m;    // tree-order point ranges
    int64_t sig_begin, n;
    int64_t u_off, v_off;    // complex128 offsets of U (3m x cap), V (3n x cap) in workspace
    int64_t g_off;           // offset of G_U = U^H U then G_V = V^H V (cap x cap each) in the
                             // Gram buffer, or -1 when the caller does not want them
    int32_t cap;             // column capacity (multiple of 3)
    int32_t pad_;
};
struct AcaResult {
    int32_t k;               // ACA rank (columns), multiple of 3
    int32_t status;          // 0 converged, 1 capacity overflow, 2 non-finite,
                             // 3 rows lost to singular pivots (block goes to the randomized SVD)
};
void launch_aca(const GreenParams& gp, const double* d_pts_p, const double* d_nrm_p,
                const AcaJob* d_jobs, int64_t njobs, double2* d_work, double2* d_gram,
                unsigned char* d_flags,
                int64_t flag_stride, double2* d_rowbuf, double2* d_colbuf, int64_t rowbuf_stride,
                int64_t colbuf_stride, double eps, AcaResult* d_res, int nctas, int capmax,
                int* d_counter, cudaStream_t st, const GreenParams* d_gps = nullptr,
                float4* d_work_df = nullptr);  // U, V as double-float pairs (then d_work may be null)
int aca_ctas_per_sm(int capmax);
// Core of the recompression for a batch: ranks r' and the k x r' transforms.
// g_off[j] >= 0: the job's Gram matrices (ld g_ld[j]) are read from d_gram instead of
// being recomputed from the factors.
// H-LU factorisation and direct solver (hlu.cu, Sec. 3.2), FP64, kept in the handle.
struct hm_matrix;
void hlu_factor(hm_matrix* h, double eps_lu, cudaStream_t st);
void hlu_solve(hm_matrix* h, int32_t nrhs, const double2* b, double2* x, cudaStream_t st);
void hlu_info(const hm_matrix* h, double* seconds, int64_t* entries, int64_t* launches);
void hlu_release(hm_matrix* h, cudaStream_t st);

// Randomized SVD (rsvd.cu) of admissible blocks the vector ACA cannot pivot.
struct RsvdBlock {
    int64_t tau_global, sig_global;  // first row / column point, tree order (batch-global)
    int64_t m, n;                    // points
    uint64_t key;                    // test-matrix key: rsvd_key of the problem-local first points
    int32_t prob;                    // problem (index into the Green parameters)
    int32_t l = 0;                   // out: samples (rank of Q)
    bool certified = false;          // out: the probes certified the range error
    int64_t u_off = 0, v_off = 0;    // out: U = Q (3m x l), V = A^H Q (3n x l) in the workspace
};
uint64_t rsvd_key(int64_t tau_begin, int64_t sigma_begin);
// Returns the FP64 factor workspace (allocated in owner) holding every block's U and V.
double2* rsvd_factors(std::vector<RsvdBlock>& blocks, const GreenParams* d_gps, const double* d_pts,
                      const double* d_nrm, double eps, std::vector<DevBuf>& owner, cudaStream_t st);

void* recompress_core(const std::vector<int64_t>& u_off, const std::vector<int64_t>& v_off,
                      const std::vector<int64_t>& m3, const std::vector<int64_t>& n3,
                      const std::vector<int32_t>& k, const std::vector<int64_t>& g_off,
                      const std::vector<int32_t>& g_ld, const double2* d_gram, int recompress,
                      double2* d_work, double eps, std::vector<int32_t>& ranks,
                      std::vector<int64_t>& s_off, cudaStream_t st);
// Writes U' = U T_U / V' = V T_V (FP32, column-major, ld = factor rows) for
// row slices: job_of[i], which[i] (0 = U, 1 = V), first row row0[i], rows[i]
// (<= 192), destination dst[i] (element offset of the slice's first row in
// d_out), ld[i] (= factor rows).  d_work_df: the double-float copy of d_work
// the ACA keeps (same offsets), read instead of converting d_work, or null.
void recompress_apply(void* batch, const std::vector<int64_t>& job_of,
                      const std::vector<int32_t>& which, const std::vector<int64_t>& row0,
                      const std::vector<int32_t>& rows, const std::vector<int64_t>& dst,
                      const std::vector<int32_t>& ld, const std::vector<int32_t>& ranks,
                      const double2* d_work, const float4* d_work_df, float2* d_out, cudaStream_t st);
void recompress_release(void* batch, cudaStream_t st);

// ---------------- rank predictor (rankmlp.cu) ----------------
void rank_model_predict_dev(const float* dP, const float* dF, int64_t n, float* dOut,
                            cudaStream_t st);
// features of an admissible block (f of the rank predictor)
void rank_features(const hm_cluster& t, const hm_cluster& s, double ks, double kp, double eps,
                   float f[6]);

// ---------------- autotuner (tune.cu) ----------------
struct hm_matrix;
// Picks the product's launch parameters for the handle: from the cache file
// at path if it holds the handle's workload key, else by timing the
// candidates on the handle and recording the best in the file (path NULL or
// empty: defaults).
void tune_product(hm_matrix* h, const char* path, cudaStream_t st);

// ---------------- GMRES (gmres.cu) ----------------
struct GmresResult {
    int iters;
    double relres;
    int converged;
};
struct hm_matrix;
GmresResult gmres_solve(hm_matrix* h, const double2* b, double2* x, int restart, double tol,
                        int maxit, cudaStream_t st);
// ||A - A_H||_F and ||A||_F (exact tensors vs the stored FP32 H-matrix) over
// every point pair (nsample <= 0) or nsample pairs drawn with the seed.
void estimate_error(hm_matrix* h, int64_t nsample, uint64_t seed, double* delta_f, double* norm_f,
                    cudaStream_t st);
// nrhs right-hand sides in lockstep (b, x: 3 nc x nrhs column-major, device)
// Independent problems of a joined handle (block-diagonal operator): one
// restarted GMRES per segment of seg_points points, in lockstep, one product
// of the whole operator per Arnoldi step (b, x: concatenated, device).
void gmres_solve_segments(hm_matrix* h, const std::vector<int64_t>& seg_points, const double2* b,
                          double2* x, int restart, double tol, int maxit,
                          std::vector<GmresResult>& out, cudaStream_t st);
void gmres_solve_multi(hm_matrix* h, int nrhs, const double2* b, double2* x, int restart, double tol,
                       int maxit, std::vector<GmresResult>& out, cudaStream_t st);

// ---------------- the handle ----------------
struct hm_matrix {
    int device = 0;
    int64_t nc = 0;
    int kernel = 0;
    double rho = 1, lam = 2, mu = 1, omega = 1, eps = 1e-4, eta = 3;
    int64_t leaf = 32;
    hm_opts opts{};
    GreenParams gp{};

    std::vector<DevBuf> owner;       // every device allocation of the handle
    double* d_pts_p = nullptr;       // tree-order points (n x 3)
    double* d_nrm_p = nullptr;       // tree-order normals (n x 3) or null
    int64_t* d_perm = nullptr;

    std::vector<int64_t> perm;
    std::vector<hm_cluster> clusters;
    std::vector<hm_block> blocks;
    int depth = 0;

    MatvecPlan plan;
    MatvecDev* mv = nullptr;
    float2* d_xp = nullptr;          // tree-order work vectors (complex64)
    float2* d_yp = nullptr;
    double2* d_xh = nullptr;         // host-API staging (complex128)
    double2* d_yh = nullptr;
    int64_t staging_cols = 0;

    // statistics
    double t_tree_ms = 0, t_part_ms = 0, t_near_ms = 0, t_aca_ms = 0, t_recomp_ms = 0,
           t_copy_ms = 0, t_total_ms = 0;
    // the layout phase in parts (host clock): storage plan, arena and item
    // tables, staged-factor copy, BF16 copy, autotuner / cache, product graph
    double t_plan_ms = 0, t_arena_ms = 0, t_stage_ms = 0, t_bf16_ms = 0, t_tune_ms = 0,
           t_graph_ms = 0;
    double apply_flops_df = 0;  // double-float flops of the factor application U' = U T_U
    int64_t aca_overflow_reruns = 0;
    int64_t aca_batches = 0;
    // device time of the ACA and recompression kernels (CUDA events on the build stream)
    double ev_aca_ms = 0, ev_recomp_ms = 0;
    // algorithmic FP64 flops of the ACA: per rank-3 step with k columns already
    // built, 18 k (m + n) complex multiply-adds (residual row and column, and the
    // Gram / cross terms of the norm update), 8 flops each
    double aca_flops = 0;
    double aca_flops_fp64 = 0;       // FP64 flops of the model (factor columns U = C gamma)
    double aca_flops_df = 0;         // double-float flops of the model on the FP32 pipes
                                     // (residuals, norm-update cross terms, Gram blocks)
    double aca_green_evals = 0;      // Green's tensors evaluated by the ACA (FP64)
    int64_t aca_workspace_peak = 0;  // largest ACA workspace of one batch (bytes)
    int64_t aca_workspace_total = 0; // ACA workspace summed over batches and re-runs (bytes)
    int batch_problems = 1;          // problems that shared the ACA / recompression launches
    int64_t rsvd_blocks = 0;       // admissible blocks compressed by the randomized SVD
    int64_t rsvd_uncertified = 0;  // of those, blocks whose samples reached their cap uncertified
    double t_rsvd_ms = 0;          // wall time of the randomized SVD pass (with its recompression)
    void* hlu = nullptr;           // H-LU factors (hlu.cu), if computed
    // autotuned product parameters (tune.cu): where they came from ("default",
    // "cache" or "sweep"), the workload key, the values and the sweep's timings
    std::string tune_source = "default", tune_key, tune_trials;
    int tune_nstage = 3;
    int64_t tune_item_bytes = 256 * 1024;
    double tune_ms = 0;
    // the last GMRES solve: fast and accurate products made, restart cycles
    int64_t gm_fast = 0, gm_accurate = 0, gm_cycles = 0;
    int used_rank_model = 0;
    // a joined batch (hm_batch_join): points of each problem, in order; empty otherwise
    std::vector<int64_t> segments;
    // two clouds (hm_build2): the number of target points, which come first (their
    // clusters too); 0 for one cloud
    int64_t n_targets = 0;
    int64_t sigma_root = 0;  // the sources' root cluster (0 for one cloud)
};

/*
 * hm.h — C ABI of the GB300 (sm_103a) H-matrix hot path for dense 3D
 * time-harmonic elastodynamic systems, after Chaillat, Desiderio & Ciarlet,
 * arXiv:1706.09384.
 *
 * The library builds, on one GPU, the H-matrix approximation A_H of the dense
 * system A p = b of Eq. (syst_a) (Sec. 1), whose 3x3 block (i, j) is the
 * Green's tensor U_w(x_i, x_j) of Eq. (elasto_U) or T_w(x_i, x_j) of
 * Eq. (elasto_T), and applies it (Sec. 3.1) inside GMRES.  Steps:
 *   cluster tree by box bisection (Sec. 2.1, "Clustering of the unknowns");
 *   block partition with the box admissibility of Eq. (admissibility_cond_bis)
 *     (Sec. 6.1) and eta (Sec. 6.2);
 *   dense near-field blocks from the Green's tensors;
 *   vector ACA with rank-3 updates and the sigma_3 pivot (Sec. 2.2 six steps
 *     and stopping test Eq. (stop_part); Sec. 2.3 strategy 3);
 *   QR + SVD recompression with eps_ACA (Sec. 3.2);
 *   H-matrix-vector product (Sec. 3.1) and restarted GMRES.
 *
 * Conventions (all entry points)
 *   - Point i owns the DOFs 3i, 3i+1, 3i+2 (point-major interleaving of the
 *     3x3 block structure, Sec. 2.3).  Vectors are complex128 (interleaved
 *     re/im doubles) of length 3*n_c in the caller's ORIGINAL point order;
 *     with nrhs > 1 they are column-major 3*n_c x nrhs.
 *   - k_s = omega sqrt(rho/mu), k_p = omega sqrt(rho/(lambda + 2 mu)) (Sec. 1).
 *     Time convention e^{+i k r} (Eq. elasto_U).
 *   - The diagonal 3x3 blocks (i = j) are opts->diag_value * I3 (the Green's
 *     tensors are singular there; the paper's collocation quadrature of that
 *     term, Sec. 4, is not part of this library).
 *   - The library copies its inputs; the caller keeps ownership of every
 *     pointer it passes.  Device pointers must be allocated on the current
 *     device; "stream" is a cudaStream_t (NULL = legacy default stream).
 *   - Every failure is reported as an hm_status; nothing aborts, no exception
 *     crosses the ABI.  After an error a handle stays valid (or is NULL when
 *     hm_build itself failed).  A handle must not be used from two host
 *     threads at once.
 *   - hm_last_error() returns a thread-local text describing the last error.
 */
#ifndef HM_H
#define HM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_matrix* hm_handle;

typedef enum { HM_KERNEL_U = 0, HM_KERNEL_T = 1 } hm_kernel;
typedef enum { HM_STORE_FP32 = 0, HM_STORE_BF16 = 1 } hm_storage;

typedef enum {
    HM_OK = 0,
    HM_ERR_ARG = 1,       /* invalid argument (null pointer, size, NaN input ...) */
    HM_ERR_CUDA = 2,      /* a CUDA call failed; see hm_last_error() */
    HM_ERR_OOM = 3,       /* device memory exhausted */
    HM_ERR_NOCONV = 4,    /* GMRES stopped at maxit above the tolerance */
    HM_ERR_TIMEOUT = 5,   /* a bounded device wait gave up */
    HM_ERR_NUMERIC = 6,   /* non-finite value produced (NaN/Inf) */
    HM_ERR_UNSUPPORTED = 7
} hm_status;

/* Build options.  Always initialise with hm_opts_default(). */
typedef struct {
    int32_t storage;          /* hm_storage for dense blocks and factors (HM_STORE_FP32) */
    int32_t aca_fp32;         /* must be 0 (HM_ERR_ARG otherwise): the ACA computes its residual
                                 rows and columns in double-float arithmetic (FP32 pairs, ~44
                                 bits) over U and V stored as double-float pairs, its pivots
                                 and norm updates in FP64; no FP32 variant exists */
    double diag_value;        /* value of the i = j blocks: diag_value * I3 (1.0) */
    double fp64_switch_ksr;   /* > 0.  Green's tensors (near field, ACA rows and columns,
                                 randomized sketches) are evaluated in FP64 where k_s r < this
                                 and in FP32 where k_s r >= this (distance and phase k r still
                                 formed in FP64).  The cancellation between the two
                                 Helmholtz terms of Eq. elasto_U costs about u / (k_s r)^2 of
                                 relative accuracy: beyond k_s r = 1 an FP32 U tensor is good to
                                 a few 1e-7 of its largest entry, a T tensor to 4e-6 (below
                                 1e-6 from k_s r = 2).  Default +inf: always FP64.
                                 hm_estimate_error always uses FP64 tensors. */
    int32_t recompress;       /* 1: QR+SVD recompression of Sec. 3.2 (default), 0: keep ACA */
    int32_t aca_max_rank;     /* initial ACA capacity in columns per block (0 = 144);
                                 blocks that need more are re-run with twice the capacity */
    int64_t workspace_bytes;  /* bound on the ACA workspace of one batch (0 = half of the
                                 device memory free when the batch is formed, counting
                                 what the library's pool holds for reuse, at least 1 GiB:
                                 fewer batches, fewer launch tails).  The workspace comes
                                 from that pool and stays reserved after the build (see
                                 hm_release_cached_memory) */
    int32_t verbose;          /* 1: phase timings on stderr */
    int32_t pad_;
    const double* weights;    /* HOST, n_c column weights w_j (NULL = 1): block (i, j), i != j,
                                 becomes K(x_i, x_j) w_j - the quadrature weights W_y of the
                                 collocation matrix A = U W_y V_y (Sec. 4) */
    const float* rank_model;  /* HOST, HM_RANK_MODEL_PARAMS floats of a trained rank predictor
                                 (see hm_rank_model_train), or NULL: when given, each admissible
                                 block's ACA workspace is sized from the predicted rank and
                                 blocks of similar predicted rank are batched together; blocks
                                 whose rank exceeds the prediction are re-run, so the H-matrix
                                 is the same either way */
    const char* tune_cache;   /* HOST path of the autotuner's cache file, or NULL (default
                                 launch parameters).  After the build, the H-matvec's launch
                                 parameters (stages of the streamed BF16 product; work-item
                                 size of the FP32 product) are read from this file for the
                                 handle's workload class (GPU, storage, leading dimension,
                                 log2 of the product's bytes), or, when the file has no such
                                 entry, picked by timing the candidates on the handle and
                                 written to it (a text file, one line per class; rewritten
                                 through a temporary file).  The parameters change only the
                                 schedule of the product.  The path is not kept after the
                                 build. */
} hm_opts;

void hm_opts_default(hm_opts* opts);

/* Builds A_H (Sec. 2-3.2) on the current device.
 *   points   host, n_c x 3 row-major FP64 (x_i = y_i, one cloud: collocation, Sec. 4)
 *   normals  host, n_c x 3 row-major FP64 unit normals n(y_j); required for
 *            HM_KERNEL_T (Eq. elasto_T acts on y), ignored (may be NULL) for U
 *   rho, lambda, mu, omega  material and circular frequency (Sec. 1), all > 0
 *   kernel   HM_KERNEL_U or HM_KERNEL_T
 *   eps      eps_ACA of Eq. (stop_part) and of the recompression (Sec. 3.2), in (0, 1)
 *   eta      eta-hat of Eq. (admissibility_cond_bis) (the paper uses 3, Sec. 6.2), > 0
 *   leaf_size  N_leaf: clusters with <= leaf_size points are not split (Sec. 2.1);
 *            1..1024 (the paper uses 100, Sec. 7).  The stored blocks are cut along
 *            segments of at most 64 points of each leaf, so larger leaves only
 *            change the tree and the partition, not the product kernels. 
 *   opts     NULL for defaults
 *   stream   cudaStream_t for all work (the call returns after the build is complete)
 *   out      receives the handle (NULL on error)
 * An admissible block whose vector ACA had to retire a row with a non-negligible
 * residual because all its 3x3 candidate pivots are singular (Sec. 2.3: T on
 * coplanar points has rank-2 3x3 blocks) is compressed by the randomized SVD
 * instead (the remark closing Sec. 2.3): an FP64 Gaussian sketch of l columns
 * (l = 64, doubling up to min(3m, 3n, 768) until 8 probe columns certify a
 * range error below eps/2), its orthonormal basis Q, V = A^H Q, then the
 * recompression with eps sqrt(3)/2; its hm_block reads rank_aca = l.  The
 * statistics count such blocks (rsvd_blocks) and those whose samples reached
 * the cap uncertified (rsvd_uncertified).
 * Errors: HM_ERR_ARG (n_c < 1, non-finite or non-positive parameters, missing
 * normals for T, non-finite coordinates, two distinct points at the same
 * position: their Green's tensor is singular), HM_ERR_OOM, HM_ERR_CUDA. */
hm_status hm_build(const double* points, const double* normals, int64_t n_c, double rho,
                   double lambda, double mu, double omega, int32_t kernel, double eps, double eta,
                   int64_t leaf_size, const hm_opts* opts, void* stream, hm_handle* out);

/* Builds the H-matrix between two clouds (Sec. 4: the collocation points x_i
 * are the rows, the integration points y_j with their normals and weights the
 * columns; Sec. 2.1: a cluster tree per cloud, the partition pairs target and
 * source clusters from the two roots with the admissibility of Sec. 6.1): the
 * rectangular A (3 n_x x 3 n_y), block (i, j) = K(x_i, y_j) w_j.  Compression,
 * randomized fallback, recompression and storage are those of hm_build.
 *   targets  host n_x x 3 FP64;  sources host n_y x 3 FP64;
 *   normals  host n_y x 3 unit normals at the sources (T kernel), else NULL;
 *   opts->weights: NULL or n_y source weights w_j.
 * The handle's index space is the n_x + n_y points, targets first: vectors
 * given to hm_matvec / hm_matvec_host have 3 (n_x + n_y) entries in the order
 * (targets, sources), each part in its cloud's original point order; the
 * product reads the source part of x (the target part is ignored) and writes
 * A x_sources into the target part of y (the source part of y is zero).
 * hm_stats reports n_targets.  hm_gmres, hm_gmres_multi (the operator is
 * rectangular), hm_lu_factor and hm_estimate_error report HM_ERR_UNSUPPORTED;
 * two-cloud handles cannot be joined.
 * Errors: HM_ERR_ARG (as hm_build; also a source point that coincides with a
 * target point: the tensor is singular there), HM_ERR_OOM, HM_ERR_CUDA. */
hm_status hm_build2(const double* targets, int64_t n_x, const double* sources,
                    const double* normals, int64_t n_y, double rho, double lambda, double mu,
                    double omega, int32_t kernel, double eps, double eta, int64_t leaf_size,
                    const hm_opts* opts, void* stream, hm_handle* out);

/* Right-hand sides per block of the tensor-core product (see hm_matvec). */
#define HM_NRHS_BLOCK 32

/* One problem of a batch build (arguments of hm_build, plus its own column
 * weights; the batch shares eps and the options). */
typedef struct {
    const double* points;   /* HOST n_c x 3 row-major */
    const double* normals;  /* HOST n_c x 3, required for the T kernel, else NULL */
    int64_t n_c;
    double rho, lambda, mu, omega;
    int32_t kernel;         /* HM_KERNEL_U or HM_KERNEL_T */
    int32_t pad_;
    double eta;
    int64_t leaf_size;
    const double* weights;  /* HOST n_c column weights w_j (W_y of Sec. 4) or NULL */
} hm_problem;

/* Builds nprob independent H-matrices at once: trees, partitions, near
 * fields and storage per problem, while the vector ACA and the recompression
 * of the admissible blocks of all problems run in shared launches (one
 * persistent ACA launch serves blocks of every problem; no paper counterpart:
 * batching of independent problems).  Each handle is the same H-matrix that
 * hm_build would give for its problem with opts.weights = probs[q].weights;
 * its statistics report the shared launches (batch_problems = nprob).
 *   probs    HOST array of nprob problems; eps and opts (NULL = defaults; its
 *            weights field is ignored) are common to the batch
 *   out      HOST array of nprob handles (all NULL on error)
 * Errors: as hm_build, for the first problem that fails. */
hm_status hm_build_batch(int32_t nprob, const hm_problem* probs, double eps, const hm_opts* opts,
                         void* stream, hm_handle* out);

/* Joins built handles into one handle whose operator is the block-diagonal
 * diag(A_1, ..., A_nprob) of their H-matrices (no paper counterpart: batching
 * of independent problems).  Vectors of the joined handle are the
 * concatenation of the problems' vectors, problem q's 3 n_c(q) entries (in its
 * original point order) after those of problems 0..q-1.  Its stored data is a
 * copy (the input handles stay valid and unchanged; free them if they are
 * not needed), laid out so that one H-matvec of the joined handle applies
 * every problem's operator in the same kernel launches.  hm_matvec,
 * hm_matvec_host, hm_gmres (one GMRES on the whole block-diagonal system),
 * hm_gmres_batch, hm_stats and the inspection calls work on it;
 * hm_estimate_error, hm_lu_factor and hm_rank_samples report
 * HM_ERR_UNSUPPORTED.  All handles must be on the current device with the
 * same storage; a joined handle cannot be joined again.
 *   hs   HOST array of nprob handles;  out: the joined handle (NULL on error)
 * Errors: HM_ERR_ARG, HM_ERR_OOM, HM_ERR_CUDA. */
hm_status hm_batch_join(int32_t nprob, const hm_handle* hs, void* stream, hm_handle* out);

/* One restarted GMRES(restart) per problem of a joined handle, run in
 * lockstep: each Arnoldi step makes one product of the block-diagonal
 * operator (all problems at once), and per-problem Gram-Schmidt, Givens
 * rotations and convergence tests (x_0 = 0, true relative residual
 * ||b_q - A_q x_q|| / ||b_q|| <= tol at restarts, accurate restart products
 * as in hm_gmres).  A problem that converges is frozen while the others go
 * on.  b, x: DEVICE complex128 concatenated vectors (see hm_batch_join), not
 * overlapping.  iters, relres: HOST arrays of nprob entries or NULL (products
 * made until each problem converged; final true relative residual).
 * Errors: HM_ERR_ARG (not a joined handle, bad arguments), HM_ERR_NOCONV
 * (some problem reached maxit), HM_ERR_TIMEOUT, HM_ERR_OOM, HM_ERR_CUDA. */
hm_status hm_gmres_batch(hm_handle h, const void* b, void* x, int32_t restart, double tol,
                         int32_t maxit, int32_t* iters, double* relres, void* stream);

/* y = A_H x (Sec. 3.1: dense product on P^non-ad, U (V^H x) on P^ad).
 *   x, y  DEVICE complex128, 3 n_c x nrhs column-major, original point order;
 *         x is read, y is overwritten; they must not overlap.
 *   nrhs  >= 1.  Work is enqueued on stream; the call does not synchronise.
 * With BF16 storage and nrhs > 1 the right-hand sides are taken in blocks of
 * HM_NRHS_BLOCK (the last one padded with zeros) and each block runs as one
 * dense contraction on the tcgen05 tensor cores: X, T = V^H X and the
 * products in BF16, sums in FP32 (relative error a few 2^-9).  Otherwise each right-hand
 * side is one product with FP32 (or BF16 x FP32) arithmetic.
 * Errors: HM_ERR_ARG (null/overlapping pointers, nrhs < 1), HM_ERR_CUDA.  With
 * BF16 storage the product kernels wait on their own shared-memory copies with
 * a time limit; a wait that gives up is reported as HM_ERR_TIMEOUT by the next
 * hm_matvec_host or hm_gmres on the handle. */
hm_status hm_matvec(hm_handle h, int32_t nrhs, const void* x, void* y, void* stream);

/* Same product with HOST buffers: x is copied to a device buffer of the handle
 * and y back, inside the call (synchronises stream before returning); the
 * result and the product's error code come back with one synchronisation.
 * Pinned host memory gives the fastest copies.  x and y must not overlap.
 * Errors as hm_matvec. */
hm_status hm_matvec_host(hm_handle h, int32_t nrhs, const void* x, void* y, void* stream);

/* Solves A_H x = b by restarted GMRES(restart) with x_0 = 0 in FP64 vectors
 * (Arnoldi by classical Gram-Schmidt with one re-orthogonalisation, complex
 * Givens rotations), stopping when the true relative residual
 * ||b - A_H x|| / ||b|| <= tol (checked at each restart with the accurate
 * product) or after maxit matvecs.  With BF16 storage each restart cycle is a
 * step of iterative refinement: its Arnoldi iteration (BF16 products) stops at
 * max(tol ||b||, delta ||r|| / 2), r the cycle's true starting residual and
 * delta the BF16 product's relative accuracy (1e-4 until a cycle measures a
 * worse one), since the true residual cannot follow the BF16 operator further.
 * b, x: DEVICE complex128, length 3 n_c, original order.
 *   iters, relres: host outputs (may be NULL).
 * Errors: HM_ERR_ARG, HM_ERR_NOCONV (maxit reached; x holds the last iterate),
 * HM_ERR_TIMEOUT (see hm_matvec), HM_ERR_CUDA. */
hm_status hm_gmres(hm_handle h, const void* b, void* x, int32_t restart, double tol,
                   int32_t maxit, int32_t* iters, double* relres, void* stream);

/* hm_gmres for nrhs right-hand sides at once: one restarted GMRES per column,
 * run in lockstep so that each Arnoldi step makes one product of all columns
 * (the tensor-core block product when the storage is BF16).  A column whose
 * residual estimate reaches its cycle's threshold (as hm_gmres) stops for the
 * rest of its cycle; restarts use the accurate product per column (iterative
 * refinement).
 *   b, x    DEVICE complex128, 3 n_c x nrhs column-major, original order; no overlap
 *   iters   HOST int32[nrhs] or NULL: products made until each column converged
 *   relres  HOST double[nrhs] or NULL: final true relative residual per column
 * Memory: (restart + 2) * nrhs vectors of 3 n_c complex128 on the device,
 * taken from a stream-ordered memory pool that the library keeps per device
 * (hm_gmres too); memory a solve frees stays reserved in that pool for the
 * next solve on any handle, until the process exits.
 * Errors: HM_ERR_ARG, HM_ERR_NOCONV (some column reached maxit; x holds the
 * last iterates), HM_ERR_TIMEOUT, HM_ERR_OOM, HM_ERR_CUDA. */
hm_status hm_gmres_multi(hm_handle h, int32_t nrhs, const void* b, void* x, int32_t restart,
                         double tol, int32_t maxit, int32_t* iters, double* relres, void* stream);

/* The approximation error of the stored H-matrix for the a-posteriori bound
 * of Sec. 3.3 (Eq. est_direct), ||b - A x|| <= ||b - A_H x|| + ||A - A_H||_F ||x||:
 *   delta_f = ||A - A_H||_F, norm_f = ||A||_F, A the exact matrix (FP64 Green's
 *   tensors, weights, diagonal blocks), A_H the stored FP32 H-matrix.
 *   nsample <= 0: every point pair (n_c <= 2048); else nsample pairs drawn
 *   uniformly by a counter-based generator from seed (unbiased estimates of
 *   the squared norms).  delta_f, norm_f: HOST outputs.  Synchronises stream.
 * Errors: HM_ERR_ARG, HM_ERR_CUDA.  (No paper counterpart for the sampling.) */
hm_status hm_estimate_error(hm_handle h, int64_t nsample, uint64_t seed, double* delta_f,
                            double* norm_f, void* stream);

/* H-LU factorisation and direct solver (Sec. 3.2, "H-LU factorization and
 * direct solver"), FP64 on the device.  hm_lu_factor copies the stored
 * H-matrix into its block tree (FP32 -> FP64) and factorises it recursively on
 * 2 x 2 block matrices (1. A11 = L11 U11, 2. U12 = L11^{-1} A12,
 * 3. L21 = A21 U11^{-1}, 4. A22 - L21 U12 = L22 U22), without pivoting; the
 * update of step 4 is formed in the target block's format and low-rank targets
 * are recompressed (Sec. 3.2) with eps_lu.  The factors replace earlier ones
 * in the handle.  Independent subtrees of the recursion run on up to 16
 * library-owned streams, each driven by a host thread of the call; they start
 * after the work already queued on stream and the call returns after all of
 * them (it synchronises stream).  The handle must not be used by another
 * thread meanwhile.  Device memory: the FP64 factors (16 bytes per stored
 * entry, lu_entries of hm_lu_info) plus temporaries of the recompressions.
 *   eps_lu  in (0, 1): the truncation tolerance eps_LU of Sec. 3.2; from 1e-5
 *           up the recompression uses the Gram form of the build's
 *           recompression, below it Householder QR of both factors
 * Errors: HM_ERR_ARG, HM_ERR_NUMERIC (zero pivot, unconverged SVD, non-finite
 * value), HM_ERR_OOM, HM_ERR_CUDA; on error the handle keeps no factors.
 * hm_lu_solve: x = U^{-1} L^{-1} b for nrhs columns; b, x DEVICE complex128,
 *   3 n_c x nrhs column-major, original point order, not overlapping.
 *   Certify it with hm_estimate_error (Eq. est_direct of Sec. 3.3).
 *   Errors: HM_ERR_ARG (no factors, bad pointers), HM_ERR_CUDA.
 * hm_lu_info: factorisation wall time (s), complex entries stored in L and U,
 *   kernel launches of the factorisation (any output may be NULL). */
hm_status hm_lu_factor(hm_handle h, double eps_lu, void* stream);
hm_status hm_lu_solve(hm_handle h, int32_t nrhs, const void* b, void* x, void* stream);
hm_status hm_lu_info(hm_handle h, double* seconds, int64_t* entries, int64_t* launches);

/* Writes a JSON object (NUL-terminated) with the build statistics: n_c, tree
 * depth, cluster and block counts, sparsity constant C_sp (Sec. 2.1), ACA
 * and recompressed ranks (as in the rank tables of Sec. 7.2), stored bytes,
 * compression tau(H) = N_s / N^2 (Sec. 7.2), phase times in ms, and the
 * products of the last hm_gmres / hm_gmres_multi on the handle (gmres_last:
 * fast products, accurate restart products, restart cycles).
 * Errors: HM_ERR_ARG (cap too small: the required size is in *needed if non-NULL). */
hm_status hm_stats(hm_handle h, char* json, size_t cap, size_t* needed);

/* ---- inspection (host copies; used to check the GPU path piece by piece) ---- */

/* One cluster of the tree T_I: points perm[begin..end) (tree order). */
typedef struct {
    int64_t begin, end;
    int64_t child0, child1;   /* cluster indices, -1 for a leaf */
    int32_t level, is_leaf;
    double lo[3], hi[3];      /* tight bounding box (Sec. 6.1) */
} hm_cluster;

/* One block tau x sigma of the partition P. */
typedef struct {
    int64_t tau, sigma;       /* cluster indices */
    int32_t admissible;       /* 1 = low rank (P^ad), 0 = dense (P^non-ad) */
    int32_t rank_aca;         /* ACA rank (multiple of 3), 0 for dense blocks */
    int32_t rank;             /* stored rank after recompression, 0 for dense blocks */
    int32_t pad_;
} hm_block;

/* Sizes of the tree and partition. */
hm_status hm_sizes(hm_handle h, int64_t* n_c, int64_t* n_clusters, int64_t* n_blocks);
/* perm[p] = original index of the point at tree position p (n_c entries, host). */
hm_status hm_get_tree(hm_handle h, int64_t* perm, hm_cluster* clusters);
hm_status hm_get_blocks(hm_handle h, hm_block* blocks);
/* Stored data of block b widened to complex128 on the host: dense block
 * (3|tau| x 3|sigma| column-major) into a, or the factors U (3|tau| x rank) into
 * a and V (3|sigma| x rank) into v, with block = U V^H; rows in tree order. */
hm_status hm_get_block_data(hm_handle h, int64_t b, void* a, void* v);

/* ---- direct kernel access ---- */

/* Evaluates K(x_q, y_q) for q = 0..npairs-1 on the GPU in FP64 (Eq. elasto_U or
 * Eq. elasto_T; for T the normal is taken at y).  x, y, ny: DEVICE npairs x 3 FP64;
 * ny may be NULL for U.  out: DEVICE npairs x 9 complex128, each 3x3 row-major.
 * Points with x_q == y_q give diag_value * I3. */
hm_status hm_green_eval(int32_t kernel, double rho, double lambda, double mu, double omega,
                        double diag_value, const double* x, const double* y, const double* ny,
                        int64_t npairs, void* out, void* stream);

/* Builds a handle from a given tree, partition and block data (host arrays, in
 * the layouts of hm_get_tree / hm_get_blocks / hm_get_block_data, block data
 * concatenated in block order: dense blocks 9|tau||sigma| entries, low-rank
 * blocks U then V), converting them to the storage precision.  Used to apply
 * an H-matrix computed elsewhere (e.g. restored from a file). */
hm_status hm_import(int64_t n_c, const int64_t* perm, int64_t n_clusters,
                    const hm_cluster* clusters, int64_t n_blocks, const hm_block* blocks,
                    const void* data, const hm_opts* opts, void* stream, hm_handle* out);

/* ---- allocation-free single-block compression ---- */

/* Largest number of points on each side of a block accepted by
 * hm_aca_block_noalloc (its fixed device scratch is sized for this). */
#define HM_NOALLOC_MAX_POINTS 8192

/* Vector ACA of one block that allocates no device memory.  The paper has no
 * counterpart: this is a service entry point for callers that cannot call
 * cudaMalloc - code whose device memory is wholly owned by another allocator
 * (a framework's caching pool that has reserved the free memory, or an
 * application held to a fixed memory budget), and latency-sensitive loops that
 * must not take the device-wide synchronisation cudaMalloc / cudaFree imply.
 * It runs the FP64-residual variant of hm_build's ACA kernel (rank-3 steps,
 * sigma_3 pivot, eps stopping test) on the block K(x_i, y_j), i < m, j < n.
 * hm_build computes its residual rows and columns in double-float arithmetic
 * over double-float copies of U and V, which would not fit the fixed scratch;
 * the two variants round differently, so near the stopping threshold their
 * ranks can differ by one rank-3 step (the products agree to about eps).
 *   x: DEVICE m x 3 FP64 row points;  y: DEVICE n x 3 FP64 column points;
 *   ny: DEVICE n x 3 unit normals at y (T kernel only, else NULL);
 *   1 <= m, n <= HM_NOALLOC_MAX_POINTS;  cap: column capacity, a multiple of 3
 *   in 3..768;  uv: DEVICE complex128 output of (3m + 3n) x cap entries,
 *   16-byte aligned: U (3m x cap, column-major) then V (3n x cap), block =
 *   U[:, :rank] V[:, :rank]^H;  rank: HOST output, the ACA rank (multiple of 3).
 * Its scratch is one fixed device array of about 3 MiB inside this library,
 * held by every GPU on which the library's module is loaded until the process
 * exits.  With CUDA's default lazy module loading that happens when the module
 * is first used on the device: for a caller that uses only this entry point,
 * inside its first call.  So make the first call on each device before another
 * allocator reserves the device's free memory (or set CUDA_MODULE_LOADING=EAGER,
 * which loads the array with the library), and before any stream capture.
 * That first call looks up the array's device address (with the device
 * current) and caches it per device ordinal; a cudaDeviceReset invalidates
 * the cached address, so do not use this entry point across a reset of the
 * device.  All calls share the array and it keeps the last call's contents;
 * each call re-initialises what must start at zero, but calls that overlap on
 * the GPU (other streams, other host threads) race on it: serialise them.  The
 * call waits for its stream to finish.
 * Errors: HM_ERR_ARG (null or misaligned pointer, sizes beyond the limits,
 * cap too small for the block's rank: *rank = -1), HM_ERR_NUMERIC,
 * HM_ERR_UNSUPPORTED (a row with a non-negligible residual whose 3x3 blocks are
 * all singular, e.g. coplanar T blocks: the vector ACA cannot pivot it and
 * hm_build compresses such blocks by the randomized SVD), HM_ERR_CUDA. */
hm_status hm_aca_block_noalloc(int32_t kernel, double rho, double lambda, double mu,
                               double omega, const double* x, int64_t m, const double* y,
                               const double* ny, int64_t n, double eps, int32_t cap, void* uv,
                               int32_t* rank, void* stream);

/* ---- learned rank predictor (no counterpart in the paper) ----
 * An MLP 6 -> 64 -> 64 -> 1 (exact GELU, FP32) predicts log(1 + rank/3) of an
 * admissible block from f = (k_s D, k_p D, dist/D, log2|tau|, log2|sigma|,
 * log10 eps), D = max of the two box diameters, dist = dist_box (Sec. 6.1); the
 * rank grows with k_s D (Sec. 5.3, Sec. 8).  Parameter block layout (floats):
 * [0,6) feature mean, [6,12) feature deviation, [12] target mean, [13] target
 * deviation, W1 (64x6 row-major), b1 (64), W2 (64x64), b2 (64), w3 (64), b3. */
#define HM_RANK_MODEL_PARAMS 4687

/* Training samples of a built handle: for each admissible block (block order)
 * the 6 features into feats (HOST, n x 6) and log(1 + rank_aca/3) into targets
 * (HOST, n).  *n receives the count; pass feats = targets = NULL to query it. */
hm_status hm_rank_samples(hm_handle h, float* feats, float* targets, int64_t* n);

/* Trains the model on the GPU by mini-batch Adam on the mean squared error of
 * the standardised target.  feats (n x 6), targets (n): DEVICE.  params: DEVICE,
 * HM_RANK_MODEL_PARAMS floats holding the initial weights; the standardisation
 * constants are computed from the data and the weights updated in place.
 * Mini-batches of `batch` samples are drawn by a counter-based hash of (seed,
 * step, position).  loss: HOST array of `steps` batch losses, or NULL.
 * Errors: HM_ERR_ARG (n < 2, steps < 0, batch < 1, lr <= 0), HM_ERR_CUDA. */
hm_status hm_rank_model_train(const float* feats, const float* targets, int64_t n,
                              int32_t steps, int32_t batch, float lr, uint64_t seed,
                              float* params, float* loss, void* stream);

/* Predictions (standardised target units) for n raw feature rows; all DEVICE. */
hm_status hm_rank_model_predict(const float* params, const float* feats, int64_t n, float* out,
                                void* stream);

/* Full-batch loss and gradient of the trainable parameters (the
 * HM_RANK_MODEL_PARAMS - 14 floats after the standardisation constants);
 * params, feats, targets, grad: DEVICE; loss: HOST or NULL. */
hm_status hm_rank_model_grad(const float* params, const float* feats, const float* targets,
                             int64_t n, float* grad, float* loss, void* stream);

/* ---- measurement ---- */

/* Runs `reps` products on internal vectors (x = 1 in tree order) and reports
 * the average device time of each kernel of the product, measured with CUDA
 * events on `stream`: ms[0] gather x, ms[1] phase 1 (t = V^H x), ms[2]
 * phase 2 (dense blocks and U t), ms[3] scatter y.  bytes[0] / bytes[1] are
 * the algorithmic bytes of phases 1 / 2 (stored entries actually used, plus
 * the x, t and y entries each phase must read or write once); bytes[2] is the
 * algorithmic byte count of one whole product (stored H-matrix + x + y).
 * Errors: HM_ERR_ARG, HM_ERR_CUDA. */
hm_status hm_profile_matvec(hm_handle h, int32_t reps, double* ms, int64_t* bytes, void* stream);

/* Same report for the tensor-core product of one block of HM_NRHS_BLOCK
 * right-hand sides (BF16 storage only): ms[0] gather X (and zero T, Y),
 * ms[1] phase 1 (T = V^H X), ms[2] rounding T to BF16 and phase 2
 * (Y = D X + U T), ms[3] scatter Y; bytes[0] is its
 * algorithmic byte count (stored BF16 entries and scales, plus X, T and Y,
 * complex64, read or written once each).
 * Errors: HM_ERR_ARG, HM_ERR_UNSUPPORTED (FP32 storage), HM_ERR_TIMEOUT,
 * HM_ERR_CUDA. */
hm_status hm_profile_matvec_multi(hm_handle h, int32_t reps, double* ms, int64_t* bytes,
                                  void* stream);

/* Number of CUDA kernels this library has launched since it was loaded. */
int64_t hm_kernel_launches(void);

/* Returns to the device the memory that the library's stream-ordered pools
 * hold for reuse: the scratch of hm_gmres / hm_gmres_multi and the build
 * workspaces of hm_build / hm_build2 / hm_build_batch (the ACA factors as
 * double-float pairs and their Gram matrices, half of the free device memory
 * at most per batch, and the staged factors), which stay reserved after a call so that the next
 * build or solve on any handle reuses them without allocating.  A build that
 * runs short of device memory returns them by itself first.  Call it with no
 * library work in flight (memory still used by queued work stays reserved).
 * Handles and their H-matrices are not affected.
 * Errors: HM_ERR_CUDA. */
hm_status hm_release_cached_memory(void);

void hm_free(hm_handle h);
const char* hm_status_string(hm_status s);
const char* hm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HM_H */

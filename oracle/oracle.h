/*
 * oracle.h — plain FP64 CPU oracle for the H-matrix hot path of
 * Chaillat, Desiderio & Ciarlet, "Theory and implementation of H-matrix based
 * iterative and direct solvers for Helmholtz and elastodynamic oscillatory
 * kernels" (arXiv:1706.09384).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that the tests, the
 * smoke check and the CPU-baseline leg of the benchmark can check the CUDA
 * path against a slow, obviously correct FP64 restatement of the paper.  The
 * product path never links, loads or calls it, and it shares no source file,
 * header, helper or table with the CUDA path.
 *
 * Conventions
 *   complex numbers are passed as interleaved (re, im) doubles;
 *   point i of the cloud owns the three DOFs 3i, 3i+1, 3i+2 (point-major
 *   interleaving, the 3x3 block structure of Sec. 2.3);
 *   a 3x3 tensor G is stored row-major: G[3*alpha + beta];
 *   matrices called "col-major" have element (r, c) at r + c*ld.
 *
 * Every function cites the section / equation of the paper it restates.
 */
#ifndef HM_ORACLE_H
#define HM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Problem definition: material (rho, lambda, mu), frequency omega, kernel
 * (0 = U_omega, Eq. elasto_U; 1 = T_omega, Eq. elasto_T), the value put on
 * the i = j diagonal 3x3 block (diag_value * I3) and optional column weights:
 * block (i, j), i != j, is K(x_i, x_j) w_j (A = K W_y, Sec. 4). */
typedef struct {
    double rho, lam, mu, omega;
    int32_t kernel;
    int32_t pad_;
    double diag_value;
    const double* weights;   /* column weights w_j (the diagonal W_y of Sec. 4), NULL = 1 */
} or_problem;

/* One node of the binary cluster tree T_I (Sec. 2.1, "Clustering"). Points
 * perm[begin..end) belong to it; lo/hi is its tight bounding box. */
typedef struct {
    int64_t begin, end;
    int64_t child0, child1;   /* -1 for a leaf */
    int64_t parent;           /* -1 for the root */
    int32_t level;            /* root = 0 */
    int32_t is_leaf;
    double lo[3], hi[3];
} or_cluster;

/* One block tau x sigma of the partition P (Sec. 2.1, "Subdivision"). */
typedef struct {
    int64_t tau, sigma;       /* cluster indices */
    int32_t admissible;       /* 1: P^ad (low rank), 0: P^non-ad (dense) */
    int32_t pad_;
} or_block;

/* --- Green's tensors (Eq. elasto_U, Eq. elasto_T, component form Sec. 5.3) */
/* Radial functions psi, chi and their r-derivatives (U = psi I + chi rr^T). */
void or_radial(double r, double rho, double lam, double mu, double omega,
               double* out8 /* psi, chi, dpsi, dchi as complex */);
/* G = K(x, y); ny = normal at y (only read for T). */
void or_green(const or_problem* pb, const double* x, const double* y,
              const double* ny, double* G18);

/* --- dense matrix A of Eq. syst_a (small clouds only) */
void or_dense_matrix(const or_problem* pb, const double* pts, const double* nrm,
                     int64_t nc, double* A /* 3nc x 3nc row-major complex */);
/* out[q] = sum_j A[rows[q], j] x[j], entries evaluated on the fly. */
void or_dense_rows_matvec(const or_problem* pb, const double* pts, const double* nrm,
                          int64_t nc, const int64_t* rows, int64_t nrows,
                          const double* x, double* out, int nthreads);

/* --- cluster tree (Sec. 2.1) and admissibility (Sec. 6.1) */
int64_t or_tree_build(const double* pts, int64_t nc, int64_t leaf,
                      int64_t* perm /* nc */, or_cluster* out /* cap >= 2 nc */);
double or_diam_box(const double* lo, const double* hi);
double or_dist_box(const double* lo1, const double* hi1, const double* lo2, const double* hi2);
int or_admissible_box(const double* lo1, const double* hi1, const double* lo2,
                      const double* hi2, double eta);
/* Exact (point-set) admissibility of Eq. admissibility_cond, O(|X||Y|). */
int or_admissible_exact(const double* X, int64_t nx, const double* Y, int64_t ny, double eta);
/* Returns the number of blocks; writes them when out != NULL. */
int64_t or_partition(const or_cluster* cl, int64_t ncl, double eta, or_block* out);

/* --- small dense linear algebra */
void or_sv3(const double* M18 /* 3x3 complex row-major */, double* s3 /* descending */);
int or_svd_jacobi(const double* A, int64_t M, int64_t N, double* s,
                  double* Uo, double* Vo);           /* col-major, M >= N */
int or_qr_householder(const double* A, int64_t M, int64_t N,
                      double* Q /* M x N */, double* R /* N x N */);

/* --- vector ACA (Sec. 2.2 six steps + Sec. 2.3 rank-3 / sigma_3 pivot) on
 * an explicit dense 3m x 3n complex matrix (row-major).  U (3m x k) and V
 * (3n x k) are returned col-major in caller buffers of capacity kcap
 * columns; returns k, or -1 if kcap is too small. */
int64_t or_aca_dense(const double* A, int64_t m, int64_t n, double eps,
                     int64_t kcap, double* U, double* V, int64_t* pivots /* 2*kcap/3 or NULL */);

/* --- recompression (Sec. 3.2): QR of U and V, SVD of R_U R_V^H, truncation. */
int64_t or_recompress(const double* U, const double* V, int64_t M, int64_t N, int64_t k,
                      double eps, double* U2, double* V2, double* svals);

/* --- randomized SVD (remark of Sec. 2.3) for blocks the vector ACA cannot
 * pivot: Gaussian sketch, orthonormal range basis, projection; l doubles from
 * 64 until 8 probe columns certify the range error (eps/2), capped at
 * min(3m, 3n, 768).  A is 3m x 3n row-major; returns l with U = Q (3m x l)
 * and V = (Q^H A)^H (3n x l) col-major, or -1 if l > lcap; *ok = 0 when the
 * cap was reached uncertified.  or_gauss: the test matrix's entry for
 * (key, counter): splitmix64 + Box-Muller, complex, E|w|^2 = 1; or_rsvd_key:
 * the key of the block whose first row / column points (tree order) are given. */
int64_t or_rsvd_dense(const double* A, int64_t m, int64_t n, double eps, uint64_t key,
                      int64_t lcap, double* U, double* V, int* ok);
void or_gauss(uint64_t key, uint64_t ctr, double* out2);
uint64_t or_splitmix64(uint64_t z); /* one output of the generator from state z - gamma */
uint64_t or_rsvd_key(int64_t tau_begin, int64_t sigma_begin);

/* --- the H-matrix (build = tree + partition + dense blocks + ACA + recompress) */
typedef struct or_hmat or_hmat;
or_hmat* or_hmat_build(const or_problem* pb, const double* pts, const double* nrm,
                       int64_t nc, double eps, double eta, int64_t leaf,
                       int recompress, int64_t sample_stride, int nthreads);
void or_hmat_free(or_hmat* h);
int64_t or_hmat_nclusters(const or_hmat* h);
void or_hmat_clusters(const or_hmat* h, or_cluster* out);
void or_hmat_perm(const or_hmat* h, int64_t* perm);
int64_t or_hmat_nblocks(const or_hmat* h);
void or_hmat_blocks(const or_hmat* h, or_block* out, int64_t* rank_aca, int64_t* rank);
/* per block: 0 dense or vector ACA, 1 randomized SVD (certified), 2 randomized
 * SVD that reached its sample cap; rank_aca holds l for the latter two */
void or_hmat_block_methods(const or_hmat* h, int32_t* out);
/* dense: D (3|tau| x 3|sigma| col-major); low rank: U (3|tau| x r), V (3|sigma| x r). */
void or_hmat_block_data(const or_hmat* h, int64_t b, double* D_or_U, double* V);
void or_hmat_matvec(const or_hmat* h, const double* x, double* y);

/* Two clouds: targets X (nx points, rows) and sources Y (ny points, columns;
 * normals nrmY for T, weights from pb at y_j); a cluster tree per cloud and
 * the partition of X x Y (Sec. 2.1); x_i = y_j gives diag_value * I3. */
typedef struct or_hmat2 or_hmat2;
void or_dense_matrix2(const or_problem* pb, const double* X, int64_t nx, const double* Y, int64_t ny,
                      const double* nrmY, double* A);
int64_t or_partition2(const or_cluster* clX, int64_t nclX, const or_cluster* clY, int64_t nclY, double eta,
                      or_block* out);
or_hmat2* or_hmat2_build(const or_problem* pb, const double* X, int64_t nx, const double* Y, int64_t ny,
                         const double* nrmY, double eps, double eta, int64_t leaf, int nthreads);
void or_hmat2_free(or_hmat2* h);
int64_t or_hmat2_nblocks(const or_hmat2* h);
void or_hmat2_blocks(const or_hmat2* h, or_block* out, int64_t* rank);
int64_t or_hmat2_nclusters(const or_hmat2* h, int side);
void or_hmat2_clusters(const or_hmat2* h, or_cluster* clX, or_cluster* clY);
void or_hmat2_matvec(const or_hmat2* h, const double* x, double* y);
double or_hmat_build_seconds(const or_hmat* h);

/* --- H-LU factorisation and direct solver (Sec. 3.2): recursive 2 x 2 block
 * LU of the H-matrix (no pivoting), updates of low-rank blocks recompressed
 * with eps_lu.  eta must be the partition's.  status: 0 ok, 1 zero pivot,
 * 2 block tree / partition mismatch.  Vectors in the original point order;
 * or_hlu_dense returns L (unit lower) and U, N x N col-major, tree order. */
typedef struct or_hlu or_hlu;
or_hlu* or_hlu_factor(const or_hmat* h, double eta, double eps_lu, int* status);
void or_hlu_free(or_hlu* f);
void or_hlu_solve(const or_hlu* f, const double* b, double* x);
void or_hlu_dense(const or_hlu* f, double* L, double* U);
double or_hlu_seconds(const or_hlu* f);
int64_t or_hlu_stored(const or_hlu* f);

/* --- restarted GMRES(m) (Sec. 3.1 drives it with the H-matvec) */
int or_gmres_hmat(const or_hmat* h, const double* b, double* x, int restart, double tol,
                  int maxit, int* iters, double* relres);
int or_gmres_dense(const double* A, int64_t n, const double* b, double* x, int restart,
                   double tol, int maxit, int* iters, double* relres);

#ifdef __cplusplus
}
#endif
#endif

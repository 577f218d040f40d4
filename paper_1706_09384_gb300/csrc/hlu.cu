// hlu.cu — H-LU factorisation and direct solver (Sec. 3.2, "H-LU
// factorization and direct solver") on the GPU, in FP64.
//
// The stored H-matrix is copied (FP32 arena -> FP64) into its block tree: a
// node is a dense block, a low-rank block U V^H, or the 2 x 2 block matrix of
// its children (the recursion of the partition, Sec. 2.1).  The factorisation
// follows the four steps of Sec. 3.2 on 2 x 2 block matrices:
//   1. A11 = L11 U11 (recursion; a dense diagonal leaf: LU without pivoting);
//   2. U12 = L11^{-1} A12;   3. L21 = A21 U11^{-1};
//   4. A22 <- A22 - L21 U12, then A22 = L22 U22 (recursion).
// The update of step 4 (the 27 format cases of A''' = A + A' A'') is formed in
// the format of the target: dense targets take dense updates, subdivided
// targets are updated child by child, low-rank targets take [U, -U_p]
// [V, V_p]^H and are recompressed (Sec. 3.2: QR of both factors, SVD of
// R_U R_V^H, truncation) with eps_LU; a product with a low-rank factor stays
// factored, (A U_b) V_b^H or U_a (B^H V_a)^H, a product of two dense or
// subdivided blocks is formed densely.  L (unit lower) and U share the tree.
// A dense update of a low-rank target of 64 or more on its smaller side is
// compressed by an adaptive randomized range finder whose residual is
// computed exactly and counted in the eps_LU budget of the truncation, so the
// result keeps the truncation bound without an SVD of the whole block.
//
// The recursion runs on the host (independent subtrees on up to 16 streams,
// each driven by its own host thread) and issues one FP64 kernel per dense
// operation: complex GEMM (32 x 32 tiles, split-K for long contractions), LU
// of a dense diagonal leaf (one CTA) and triangular solves with it (a warp per
// column).  A recompression forms the k x k core W = R_U R_V^H (Householder
// QR of both factors, or for eps_LU >= 1e-5 the Gram form: Cholesky of the
// Gram matrices, no orthonormal factors), reduces W by a column-pivoted QR
// (one CTA, shared memory) and runs a one-sided block Jacobi on R^H across an
// 8-CTA cluster; its singular values are read back to choose the rank and
// size the next operation.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <exception>
#include <map>
#include <thread>
#include <vector>

#include <cooperative_groups.h>

#include "hm_internal.h"

namespace {

constexpr int HT = 256;
constexpr int TT = 32;  // GEMM tile
constexpr int TK = 16;  // GEMM K step

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ void zmad(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// C (M x N, ldc) += alpha opA(A) opB(B); op 0: X, op 1: X^H.  Split-K: CTA
// row y of the grid takes k in [y kchunk, (y + 1) kchunk) and adds into
// C + y cstride (the caller sums the partial products).
__global__ void __launch_bounds__(HT) hz_gemm_kernel(double2* C, const double2* A, const double2* B,
                                                     int64_t M, int64_t N, int64_t K, int64_t lda,
                                                     int64_t ldb, int64_t ldc, int opa, int opb,
                                                     double2 alpha, int64_t kchunk, int64_t cstride) {
    __shared__ double2 sa[TK][TT + 1];
    __shared__ double2 sb[TK][TT + 1];
    const int64_t tm = (M + TT - 1) / TT;
    const int64_t r0 = (blockIdx.x % tm) * TT, c0 = (blockIdx.x / tm) * TT;
    const int tid = threadIdx.x, tr = tid % 16, tc = tid / 16;
    const int64_t kb = blockIdx.y * kchunk, ke = min(K, kb + kchunk);
    C += blockIdx.y * cstride;
    double2 acc[2][2] = {};
    for (int64_t k0 = kb; k0 < ke; k0 += TK) {
        for (int e = tid; e < TK * TT; e += HT) {
            {  // opA(A)(r0 + rr, k0 + kk), the stored matrix's contiguous index fastest
                const int kk = opa ? e % TK : e / TT, rr = opa ? e / TK : e % TT;
                const int64_t r = r0 + rr, k = k0 + kk;
                double2 v = make_double2(0.0, 0.0);
                if (r < M && k < ke) v = opa ? zconj(A[k + r * lda]) : A[r + k * lda];
                sa[kk][rr] = v;
            }
            {  // opB(B)(k0 + kk, c0 + cc)
                const int kk = opb ? e / TT : e % TK, cc = opb ? e % TT : e / TK;
                const int64_t k = k0 + kk, c = c0 + cc;
                double2 v = make_double2(0.0, 0.0);
                if (k < ke && c < N) v = opb ? zconj(B[c + k * ldb]) : B[k + c * ldb];
                sb[kk][cc] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            const double2 a0 = sa[kk][tr], a1 = sa[kk][tr + 16];
            const double2 b0 = sb[kk][tc], b1 = sb[kk][tc + 16];
            zmad(acc[0][0], a0, b0);
            zmad(acc[0][1], a0, b1);
            zmad(acc[1][0], a1, b0);
            zmad(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int64_t r = r0 + tr + 16 * i, c = c0 + tc + 16 * j;
            if (r < M && c < N) {
                double2& d = C[r + c * ldc];
                const double2 v = zmul(alpha, acc[i][j]);
                d.x += v.x;
                d.y += v.y;
            }
        }
}

// dst (rows x cols, ldd) = alpha src (lds), or += when add
__global__ void hz_copy_kernel(double2* dst, int64_t ldd, const double2* src, int64_t lds, int64_t rows,
                               int64_t cols, double2 alpha, int add) {
    const int64_t ne = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)HT + threadIdx.x; e < ne; e += (int64_t)gridDim.x * HT) {
        const int64_t r = e % rows, c = e / rows;
        const double2 v = zmul(alpha, src[r + c * lds]);
        double2& d = dst[r + c * ldd];
        if (add) {
            d.x += v.x;
            d.y += v.y;
        } else {
            d = v;
        }
    }
}

// C (rows x cols, ldc) += sum over the splits of P (rows x cols each, in order)
__global__ void hz_splitsum_kernel(double2* C, int64_t ldc, const double2* P, int64_t rows, int64_t cols,
                                   int64_t splits) {
    for (int64_t e = blockIdx.x * (int64_t)HT + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * HT) {
        double2 a = make_double2(0.0, 0.0);
        for (int64_t q = 0; q < splits; ++q) {
            a.x += P[q * rows * cols + e].x;
            a.y += P[q * rows * cols + e].y;
        }
        double2& d = C[e % rows + (e / rows) * ldc];
        d.x += a.x;
        d.y += a.y;
    }
}

__global__ void hz_identity_kernel(double2* A, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)HT + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * HT)
        A[e] = make_double2((e % n) == (e / n) ? 1.0 : 0.0, 0.0);
}

// LU without pivoting of a dense m x m block, in place (one CTA).
__global__ void __launch_bounds__(HT) hz_getrf_kernel(double2* D, int64_t m, int* zero_pivot) {
    for (int64_t p = 0; p < m; ++p) {
        const double2 piv = D[p + p * m];
        if (piv.x == 0.0 && piv.y == 0.0) {
            if (threadIdx.x == 0) atomicOr(zero_pivot, 1);
            return;  // uniform across the CTA
        }
        for (int64_t r = p + 1 + threadIdx.x; r < m; r += HT) D[r + p * m] = zdiv(D[r + p * m], piv);
        __syncthreads();
        const int64_t w = m - p - 1;
        for (int64_t e = threadIdx.x; e < w * w; e += HT) {
            const int64_t r = p + 1 + e % w, c = p + 1 + e / w;
            const double2 l = D[r + p * m], u = D[p + c * m];
            D[r + c * m].x -= l.x * u.x - l.y * u.y;
            D[r + c * m].y -= l.x * u.y + l.y * u.x;
        }
        __syncthreads();
    }
}

// Triangular solves with a dense factored leaf D (m x m) on B (m x c, ldb): a
// warp per column, the column in shared memory, right-looking (once y_r is
// final it is subtracted from the rows it couples to, a lane per row).
// mode 0: L (unit lower) y = b; 1: U y = b; 2: U^H y = b.
constexpr int TW = 4;  // columns (warps) per CTA
__global__ void __launch_bounds__(TW * 32) hz_trsm_kernel(const double2* D, int64_t m, double2* B,
                                                          int64_t ldb, int64_t c, int mode) {
    extern __shared__ double2 hz_col[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double2* y = hz_col + warp * m;
    for (int64_t j = blockIdx.x * (int64_t)TW + warp; j < c; j += (int64_t)gridDim.x * TW) {
        double2* b = B + j * ldb;
        for (int64_t q = lane; q < m; q += 32) y[q] = b[q];
        __syncwarp();
        if (mode == 0) {
            for (int64_t r = 0; r < m; ++r) {
                const double2 yr = y[r];
                for (int64_t q = r + 1 + lane; q < m; q += 32) {
                    const double2 t = zmul(D[q + r * m], yr);
                    y[q].x -= t.x;
                    y[q].y -= t.y;
                }
                __syncwarp();
            }
        } else if (mode == 1) {
            for (int64_t r = m - 1; r >= 0; --r) {
                const double2 yr = zdiv(y[r], D[r + r * m]);
                __syncwarp();
                if (lane == 0) y[r] = yr;
                for (int64_t q = lane; q < r; q += 32) {
                    const double2 t = zmul(D[q + r * m], yr);
                    y[q].x -= t.x;
                    y[q].y -= t.y;
                }
                __syncwarp();
            }
        } else {
            for (int64_t r = 0; r < m; ++r) {
                const double2 yr = zdiv(y[r], zconj(D[r + r * m]));
                __syncwarp();
                if (lane == 0) y[r] = yr;
                for (int64_t q = r + 1 + lane; q < m; q += 32) {
                    const double2 t = zmul(zconj(D[r + q * m]), yr);
                    y[q].x -= t.x;
                    y[q].y -= t.y;
                }
                __syncwarp();
            }
        }
        for (int64_t q = lane; q < m; q += 32) b[q] = y[q];
        __syncwarp();
    }
}

template <int NT>
__device__ double hz_block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    return s;
}

// y_c -= tau v (v^H y_c) for columns [c_begin, c_end) of Y, rows k .. M - 1 (a warp per column)
template <int NT>
__device__ void hz_reflect(const double2* v, double tau, int64_t k, int64_t M, double2* Y, int64_t ldy,
                           int64_t c_begin, int64_t c_end) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c = c_begin + warp; c < c_end; c += NT / 32) {
        double2* y = Y + c * ldy;
        double2 w = make_double2(0.0, 0.0);
        for (int64_t r = k + lane; r < M; r += 32) {
            const double2 a = v[r], b = y[r];
            w.x += a.x * b.x + a.y * b.y;
            w.y += a.x * b.y - a.y * b.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
            w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
        }
        w.x *= tau;
        w.y *= tau;
        for (int64_t r = k + lane; r < M; r += 32) {
            const double2 a = v[r];
            y[r].x -= a.x * w.x - a.y * w.y;
            y[r].y -= a.x * w.y + a.y * w.x;
        }
    }
}

// Householder QR of W (M x K, M >= K, overwritten by the reflectors): Q (M x K)
// and R (K x K, upper).  One CTA; tau in dynamic shared memory.
constexpr int QT = 512;
__global__ void __launch_bounds__(QT) hz_qr_kernel(double2* W, int64_t M, int64_t K, double2* Q,
                                                   double2* R) {
    extern __shared__ double hz_tau[];
    __shared__ double red[QT / 32];
    for (int64_t k = 0; k < K; ++k) {
        double2* x = W + k * M;
        double s = 0.0;
        for (int64_t r = k + threadIdx.x; r < M; r += QT) s += x[r].x * x[r].x + x[r].y * x[r].y;
        const double nx2 = hz_block_sum<QT>(s, red);
        double tau = 0.0;
        double2 alpha = make_double2(0.0, 0.0);
        if (nx2 > 0.0) {
            const double2 x0 = x[k];
            const double a0 = sqrt(x0.x * x0.x + x0.y * x0.y), nx = sqrt(nx2);
            const double2 ph = a0 > 0.0 ? make_double2(x0.x / a0, x0.y / a0) : make_double2(1.0, 0.0);
            alpha = make_double2(-ph.x * nx, -ph.y * nx);  // H x = alpha e_1
            const double2 v0 = make_double2(x0.x - alpha.x, x0.y - alpha.y);
            const double vn2 = nx2 - a0 * a0 + (v0.x * v0.x + v0.y * v0.y);
            tau = 2.0 / vn2;
            __syncthreads();
            if (threadIdx.x == 0) x[k] = v0;
        }
        if (threadIdx.x == 0) {
            hz_tau[k] = tau;
            R[k + k * K] = tau != 0.0 ? alpha : make_double2(0.0, 0.0);
        }
        __syncthreads();
        if (tau != 0.0) hz_reflect<QT>(x, tau, k, M, W, M, k + 1, K);
        __syncthreads();
        for (int64_t c = k + 1 + threadIdx.x; c < K; c += QT) R[k + c * K] = W[k + c * M];  // row k of R
        for (int64_t c = threadIdx.x; c < k; c += QT) R[k + c * K] = make_double2(0.0, 0.0);
        __syncthreads();
    }
    for (int64_t e = threadIdx.x; e < M * K; e += QT)
        Q[e] = make_double2((e % M) == (e / M) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int64_t k = K - 1; k >= 0; --k) {
        if (hz_tau[k] != 0.0) hz_reflect<QT>(W + k * M, hz_tau[k], k, M, Q, M, k, K);
        __syncthreads();
    }
}

// One-sided Jacobi (Hestenes) on W0 (K x K): WJ = W0 J with mutually
// orthogonal columns P_j s_j, s_j = |WJ_j|; J (the right singular vectors) is
// not kept.  Round-robin pairs, a warp per pair; a pair is rotated when
// |gamma| > tol sqrt(alpha beta), tol = max(tol_min, K u), and neither column
// is negligible (squared norm above (K u)^2 ||W||_F^2).  One CTA working in WJ
// (global memory, L2-resident): the form for cores too large for the cluster
// kernel below.
constexpr int JT = 512;
constexpr int64_t JS_MAX_CHOL = 1024;  // Gram-form recompression: K up to here
constexpr int64_t QP_SMEM = 112;       // one-CTA cores in shared memory (K x K complex) up to here
__global__ void __launch_bounds__(JT) hz_jacobi_kernel(const double2* W0, double2* WJ, int64_t K, double* s,
                                                       int* unconverged, double tol_min) {
    __shared__ int s_conv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double2* W = WJ;
    __shared__ double red[JT / 32];
    double f2 = 0.0;
    for (int64_t e = threadIdx.x; e < K * K; e += JT) {
        const double2 v = W0[e];
        W[e] = v;
        f2 += v.x * v.x + v.y * v.y;
    }
    f2 = hz_block_sum<JT>(f2, red);  // ||W||_F^2, invariant under the rotations
    const int64_t np = (K + 1) & ~1;
    // the rounding level of the computed gamma over K terms (Demmel and Veselic 1992)
    const double tol = fmax(tol_min, (double)K * 0x1.0p-53);
    // a column at the rounding level of W (rank-deficient W) cannot be made
    // orthogonal to a large one to relative accuracy: it is left alone, and
    // its singular value (<= K u ||W||_F) falls below any truncation
    const double small = ((double)K * 0x1.0p-53) * ((double)K * 0x1.0p-53) * f2;
    int sweep = 0;
    for (; sweep < 80; ++sweep) {
        if (threadIdx.x == 0) s_conv = 1;
        __syncthreads();
        for (int64_t round = 0; round < np - 1; ++round) {
            for (int64_t pi = warp; pi < np / 2; pi += JT / 32) {
                int64_t a, b;
                if (pi == 0) {
                    a = np - 1;
                    b = round;
                } else {
                    a = (round + pi) % (np - 1);
                    b = (round - pi + np - 1) % (np - 1);
                }
                if (a >= K || b >= K) continue;
                if (a > b) {
                    const int64_t t = a;
                    a = b;
                    b = t;
                }
                double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
                for (int64_t r = lane; r < K; r += 32) {
                    const double2 wa = W[r + a * K], wb = W[r + b * K];
                    al += wa.x * wa.x + wa.y * wa.y;
                    be += wb.x * wb.x + wb.y * wb.y;
                    gr += wa.x * wb.x + wa.y * wb.y;  // conj(wa) wb
                    gi += wa.x * wb.y - wa.y * wb.x;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    gr += __shfl_xor_sync(0xffffffffu, gr, o);
                    gi += __shfl_xor_sync(0xffffffffu, gi, o);
                }
                const double ag = sqrt(gr * gr + gi * gi);
                if (al <= small || be <= small) continue;                      // uniform within the warp
                if (ag == 0.0 || ag <= tol * sqrt(al) * sqrt(be)) continue;  // uniform within the warp
                if (lane == 0) s_conv = 0;
                const double2 phc = make_double2(gr / ag, -gi / ag);  // e^{-i phi}
                const double zeta = (be - al) / (2.0 * ag);
                const double az = fabs(zeta);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (az > 1e150 ? 2.0 * az : az + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                // [w_a, w_b] <- [w_a, w_b] [[c, sn], [-sn e^{-i phi}, c e^{-i phi}]]
                for (int64_t r = lane; r < K; r += 32) {
                    const double2 wa = W[r + a * K], pwb = zmul(phc, W[r + b * K]);
                    W[r + a * K] = make_double2(c * wa.x - sn * pwb.x, c * wa.y - sn * pwb.y);
                    W[r + b * K] = make_double2(sn * wa.x + c * pwb.x, sn * wa.y + c * pwb.y);
                }
            }
            __syncthreads();
        }
        if (s_conv) break;
        __syncthreads();
    }
    if (threadIdx.x == 0 && sweep == 80) atomicOr(unconverged, 2);
    for (int64_t j = warp; j < K; j += JT / 32) {
        double a = 0.0;
        for (int64_t r = lane; r < K; r += 32) a += W[r + j * K].x * W[r + j * K].x + W[r + j * K].y * W[r + j * K].y;
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) s[j] = sqrt(a);
    }
}

// The same one-sided Jacobi as a block Jacobi on a thread-block cluster of CJ
// CTAs (one SM each, for CJ times the FP64 rate of one SM).  The K columns form
// NBJ = 2 CJ blocks of bs = ceil(K / NBJ); in a block round CTA i holds the two
// blocks of pair i of a round-robin tournament over the blocks (NBJ - 1 block
// rounds make a sweep of all block pairs) in its own shared memory and rotates
// all pairs across them, in bs rounds of disjoint pairs under CTA barriers
// (the pairs inside each block in the first block round of a sweep).  Between
// block rounds every CTA pulls its next two blocks from the CTAs that held them
// through distributed shared memory (double-buffered); the cluster barrier
// ends a block round.  A warp holds its pair of columns in registers (K <= 128).
constexpr int CJ = 8;
constexpr int CJT = 256;
constexpr int NBJ = 2 * CJ;
constexpr int64_t CJ_MAX = 128;

__device__ __forceinline__ void hz_tour(int rho, int i, int& a, int& b) {
    if (i == 0) {
        a = NBJ - 1;
        b = rho;
    } else {
        a = (rho + i) % (NBJ - 1);
        b = (rho - i + NBJ - 1) % (NBJ - 1);
    }
}

// One rotation of the pair (ca, cb) of K-long columns by a warp; true if rotated.
__device__ __forceinline__ bool hz_rot_pair(double2* ca, double2* cb, int64_t K, double tol, double small,
                                            int lane) {
    double2 wa[4], wb[4];
    double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = lane + 32 * i;
        wa[i] = r < K ? ca[r] : make_double2(0.0, 0.0);
        wb[i] = r < K ? cb[r] : make_double2(0.0, 0.0);
        al += wa[i].x * wa[i].x + wa[i].y * wa[i].y;
        be += wb[i].x * wb[i].x + wb[i].y * wb[i].y;
        gr += wa[i].x * wb[i].x + wa[i].y * wb[i].y;  // conj(wa) wb
        gi += wa[i].x * wb[i].y - wa[i].y * wb[i].x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        gr += __shfl_xor_sync(0xffffffffu, gr, o);
        gi += __shfl_xor_sync(0xffffffffu, gi, o);
    }
    const double ag = sqrt(gr * gr + gi * gi);
    if (al <= small || be <= small) return false;                      // uniform within the warp
    if (ag == 0.0 || ag <= tol * sqrt(al) * sqrt(be)) return false;  // uniform within the warp
    const double2 phc = make_double2(gr / ag, -gi / ag);  // e^{-i phi}
    const double zeta = (be - al) / (2.0 * ag);
    const double az = fabs(zeta);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (az > 1e150 ? 2.0 * az : az + sqrt(1.0 + zeta * zeta));
    const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
    // [w_a, w_b] <- [w_a, w_b] [[c, sn], [-sn e^{-i phi}, c e^{-i phi}]]
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = lane + 32 * i;
        if (r < K) {
            const double2 pwb = zmul(phc, wb[i]);
            ca[r] = make_double2(c * wa[i].x - sn * pwb.x, c * wa[i].y - sn * pwb.y);
            cb[r] = make_double2(sn * wa[i].x + c * pwb.x, sn * wa[i].y + c * pwb.y);
        }
    }
    return true;
}

__global__ void __cluster_dims__(CJ, 1, 1) __launch_bounds__(CJT)
    hz_jacobi_cluster_kernel(const double2* W0, double2* WJ, int64_t K, double* s, int* unconverged,
                             double tol_min) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double2 hz_cw[];  // [parity 2][slot 2][bs][K]
    __shared__ double part[CJ];
    __shared__ double red[CJT / 32];
    __shared__ int conv;
    const int rank = (int)cl.block_rank();
    double* part0 = cl.map_shared_rank(part, 0);
    int* conv0 = cl.map_shared_rank(&conv, 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t bs = (K + NBJ - 1) / NBJ;
    auto slot = [&](int par, int sl) { return hz_cw + (int64_t)(par * 2 + sl) * bs * K; };
    auto ncols = [&](int beta) { return (int)max((int64_t)0, min(bs, K - beta * bs)); };
    // ||W||_F^2 from slices of W0
    double f2 = 0.0;
    for (int64_t e = (int64_t)rank * CJT + threadIdx.x; e < K * K; e += (int64_t)CJ * CJT) {
        const double2 v = W0[e];
        f2 += v.x * v.x + v.y * v.y;
    }
    f2 = hz_block_sum<CJT>(f2, red);
    if (threadIdx.x == 0) part0[rank] = f2;
    // the first placement straight from W0
    {
        int A, B;
        hz_tour(0, rank, A, B);
        const int beta[2] = {A, B};
        for (int sl = 0; sl < 2; ++sl) {
            double2* dst = slot(0, sl);
            const int64_t n = (int64_t)ncols(beta[sl]) * K;
            const double2* src = W0 + (int64_t)beta[sl] * bs * K;
            for (int64_t e = threadIdx.x; e < n; e += CJT) dst[e] = src[e];
        }
    }
    cl.sync();
    f2 = 0.0;
    for (int q = 0; q < CJ; ++q) f2 += part0[q];
    const double tol = fmax(tol_min, (double)K * 0x1.0p-53);
    // a column at the rounding level of W (rank-deficient W) cannot be made
    // orthogonal to a large one to relative accuracy: it is left alone
    const double small = ((double)K * 0x1.0p-53) * ((double)K * 0x1.0p-53) * f2;
    int64_t g = 0;  // block rounds done
    int sweep = 0;
    for (; sweep < 80; ++sweep) {
        if (rank == 0 && threadIdx.x == 0) *conv0 = 1;
        cl.sync();
        for (int rho = 0; rho < NBJ - 1; ++rho, ++g) {
            const int par = (int)(g & 1);
            int A, B;
            hz_tour(rho, rank, A, B);
            if (g > 0) {  // pull both blocks from where they were in the previous block round
                const int prho = (int)((g - 1) % (NBJ - 1));
                const int beta[2] = {A, B};
                for (int sl = 0; sl < 2; ++sl) {
                    int src_cta = 0, src_sl = 0;
                    for (int j = 0; j < CJ; ++j) {
                        int a2, b2;
                        hz_tour(prho, j, a2, b2);
                        if (a2 == beta[sl]) {
                            src_cta = j;
                            src_sl = 0;
                        }
                        if (b2 == beta[sl]) {
                            src_cta = j;
                            src_sl = 1;
                        }
                    }
                    const double2* src = cl.map_shared_rank(slot(par ^ 1, src_sl), src_cta);
                    double2* dst = slot(par, sl);
                    const int64_t n = (int64_t)ncols(beta[sl]) * K;
                    for (int64_t e = threadIdx.x; e < n; e += CJT) dst[e] = src[e];
                }
                __syncthreads();
            }
            double2* SA = slot(par, 0);
            double2* SB = slot(par, 1);
            const int na = ncols(A), nb = ncols(B);
            if (rho == 0) {  // the pairs inside each block, round robin, warps 0-3 on A and 4-7 on B
                const int sl = warp / 4, p = warp % 4;
                const int n = sl == 0 ? na : nb;
                const int npl = (n + 1) & ~1;
                double2* S = sl == 0 ? SA : SB;
                const int rounds = (int)((bs + 1) & ~1) - 1;
                for (int r = 0; r < rounds; ++r) {
                    if (r < npl - 1 && p < npl / 2) {
                        int x, y;
                        if (p == 0) {
                            x = npl - 1;
                            y = r;
                        } else {
                            x = (r + p) % (npl - 1);
                            y = (r - p + npl - 1) % (npl - 1);
                        }
                        if (x < n && y < n) {
                            if (x > y) {
                                const int t = x;
                                x = y;
                                y = t;
                            }
                            if (hz_rot_pair(S + (int64_t)x * K, S + (int64_t)y * K, K, tol, small, lane) && lane == 0)
                                *conv0 = 0;
                        }
                    }
                    __syncthreads();
                }
            }
            for (int64_t r = 0; r < bs; ++r) {  // the pairs across the two blocks: (q, q + r mod bs)
                for (int64_t q = warp; q < bs; q += CJT / 32) {
                    const int64_t qb = (q + r) % bs;
                    if (q < na && qb < nb &&
                        hz_rot_pair(SA + q * K, SB + qb * K, K, tol, small, lane) && lane == 0)
                        *conv0 = 0;
                }
                __syncthreads();
            }
            cl.sync();  // this round's blocks are final before anyone pulls them
        }
        const int done = *conv0;
        cl.sync();  // every thread has read the flag before CTA 0 resets it
        if (done) break;
    }
    if (rank == 0 && threadIdx.x == 0 && sweep == 80) atomicOr(unconverged, 2);
    {  // the blocks this CTA held in the last block round, back to their columns
        const int par = (int)((g - 1) & 1);
        int A, B;
        hz_tour((int)((g - 1) % (NBJ - 1)), rank, A, B);
        const int beta[2] = {A, B};
        for (int sl = 0; sl < 2; ++sl) {
            const double2* S = slot(par, sl);
            const int n = ncols(beta[sl]);
            for (int q = warp; q < n; q += CJT / 32) {
                const int64_t j = (int64_t)beta[sl] * bs + q;
                double a = 0.0;
                for (int64_t r = lane; r < K; r += 32) {
                    const double2 v = S[q * K + r];
                    WJ[r + j * K] = v;
                    a += v.x * v.x + v.y * v.y;
                }
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) s[j] = sqrt(a);
            }
        }
    }
    cl.sync();
}

// G = R^H R for a Hermitian semi-definite G (K x K, in place -> R upper):
// equilibrated (G' = D^-1 G D^-1, D = sqrt diag G), right-looking on the upper
// triangle; a pivot of G' at or below 1e-13 zeroes its row of R (the
// direction is below 3.2e-7 of its column norm).  R = R' D.
__device__ void hz_chol_equil(double2* Gg, int64_t K, double* dsc, double2* sbuf) {
    __shared__ double s_piv;
    const int tid = threadIdx.x;
    double2* G = sbuf ? sbuf : Gg;  // the factorisation runs in shared memory when it fits
    if (sbuf) {
        for (int64_t e = tid; e < K * K; e += JT) sbuf[e] = Gg[e];
        __syncthreads();
    }
    for (int64_t j = tid; j < K; j += JT) {
        const double d = G[j + j * K].x;
        dsc[j] = d > 1e-280 ? sqrt(d) : 0.0;  // a column whose squared norm underflows counts as zero
    }
    __syncthreads();
    for (int64_t e = tid; e < K * K; e += JT) {
        const int64_t p = e % K, c = e / K;
        const double sc = (dsc[p] > 0.0 && dsc[c] > 0.0) ? 1.0 / (dsc[p] * dsc[c]) : 0.0;
        G[e] = make_double2(G[e].x * sc, G[e].y * sc);
    }
    __syncthreads();
    for (int64_t j = 0; j < K; ++j) {
        if (tid == 0) {
            const double d = G[j + j * K].x;
            s_piv = d > 1e-13 ? sqrt(d) : 0.0;
        }
        __syncthreads();
        const double piv = s_piv;
        for (int64_t c = j + 1 + tid; c < K; c += JT) {
            const double2 g = G[j + c * K];
            G[j + c * K] = piv > 0.0 ? make_double2(g.x / piv, g.y / piv) : make_double2(0.0, 0.0);
        }
        if (tid == 0) G[j + j * K] = make_double2(piv, 0.0);
        __syncthreads();
        const int64_t w = K - j - 1;
        for (int64_t e = tid; e < w * w; e += JT) {
            const int64_t a = j + 1 + e % w, b = j + 1 + e / w;
            if (a <= b) {
                const double2 ra = G[j + a * K], rb = G[j + b * K];
                G[a + b * K].x -= ra.x * rb.x + ra.y * rb.y;  // conj(ra) rb
                G[a + b * K].y -= ra.x * rb.y - ra.y * rb.x;
            }
        }
        __syncthreads();
    }
    for (int64_t e = tid; e < K * K; e += JT) {
        const int64_t p = e % K, c = e / K;
        Gg[e] = p > c ? make_double2(0.0, 0.0) : make_double2(G[e].x * dsc[c], G[e].y * dsc[c]);
    }
    __syncthreads();
}

// Core of the Gram-form recompression (one CTA): R_U, R_V from G_U = U^H U and
// G_V = V^H V (in place) and W = R_U R_V^H.
__global__ void __launch_bounds__(JT) hz_gram_core_kernel(double2* GU, double2* GV, double2* W, int64_t K) {
    extern __shared__ double2 hz_ga[];
    __shared__ double dsc[JS_MAX_CHOL];
    double2* sbuf = K <= QP_SMEM ? hz_ga : nullptr;
    hz_chol_equil(GU, K, dsc, sbuf);
    hz_chol_equil(GV, K, dsc, sbuf);
    for (int64_t e = threadIdx.x; e < K * K; e += JT) {  // W_pc = sum_q RU_pq conj(RV_cq), q >= max(p, c)
        const int64_t p = e % K, c = e / K;
        double2 a = make_double2(0.0, 0.0);
        for (int64_t q = p > c ? p : c; q < K; ++q) zmad(a, GU[p + q * K], zconj(GV[c + q * K]));
        W[e] = a;
    }
}

// Householder QR with column pivoting of W (K x K; Businger and Golub 1965):
// W Pi = Q R, the column of largest remaining norm first (ties: lowest index),
// norms recomputed at each step.  Writes R^H (K x K) and perm (Pi's column k
// is e_perm[k]); Q is not formed; the reduction stops once the largest
// remaining column is at the rounding level of W.  One CTA working in shared
// memory (K <= QP_SMEM; else in the K x K workspace Ag).  R^H is
// the preconditioned start of the one-sided Jacobi (Drmac and Veselic 2008):
// its columns are close to orthogonal, so far fewer sweeps are needed.
constexpr int64_t QP_MAX = 1024;
__global__ void __launch_bounds__(JT) hz_qrcp_kernel(const double2* W0, double2* Ag, double2* RH, int32_t* perm,
                                                     int64_t K) {
    extern __shared__ double2 hz_qa[];
    double2* A = K <= QP_SMEM ? hz_qa : Ag;
    __shared__ double cn[QP_MAX];
    __shared__ double2 alph[QP_MAX];
    __shared__ double redv[JT / 32];
    __shared__ int redi[JT / 32];
    __shared__ int s_piv;
    __shared__ double red[JT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double f2 = 0.0;
    for (int64_t e = tid; e < K * K; e += JT) {
        const double2 v = W0[e];
        A[e] = v;
        f2 += v.x * v.x + v.y * v.y;
    }
    for (int64_t j = tid; j < K; j += JT) perm[j] = (int32_t)j;
    f2 = hz_block_sum<JT>(f2, red);
    // columns at the rounding level of W are not reduced further: their
    // reflectors would divide by underflowing norms, and their part of R
    // (<= K u ||W||_F) lies below any truncation
    const double negl = ((double)K * 0x1.0p-53) * ((double)K * 0x1.0p-53) * f2;
    int64_t kstop = K;
    for (int64_t k = 0; k < K; ++k) {
        for (int64_t j = k + warp; j < K; j += JT / 32) {  // norms of the trailing columns, rows k..K-1
            double a = 0.0;
            for (int64_t r = k + lane; r < K; r += 32) a += A[r + j * K].x * A[r + j * K].x + A[r + j * K].y * A[r + j * K].y;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) cn[j] = a;
        }
        __syncthreads();
        double bv = -1.0;
        int bi = (int)k;
        for (int64_t j = k + tid; j < K; j += JT)
            if (cn[j] > bv) {
                bv = cn[j];
                bi = (int)j;
            }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            redv[warp] = bv;
            redi[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double v = redv[0];
            int i = redi[0];
            for (int w = 1; w < JT / 32; ++w)
                if (redv[w] > v || (redv[w] == v && redi[w] < i)) {
                    v = redv[w];
                    i = redi[w];
                }
            s_piv = i;
        }
        __syncthreads();
        const int64_t p = s_piv;
        if (p != k) {
            for (int64_t r = tid; r < K; r += JT) {
                const double2 t = A[r + k * K];
                A[r + k * K] = A[r + p * K];
                A[r + p * K] = t;
            }
            if (tid == 0) {
                const int32_t t = perm[k];
                perm[k] = perm[p];
                perm[p] = t;
                const double c = cn[k];
                cn[k] = cn[p];
                cn[p] = c;
            }
        }
        __syncthreads();
        double2* x = A + k * K;
        const double nx2 = cn[k];  // the largest remaining column (uniform)
        if (!(nx2 > negl)) {
            kstop = k;
            break;
        }
        double tau = 0.0;
        double2 alpha = make_double2(0.0, 0.0);
        {
            const double2 x0 = x[k];
            const double a0 = sqrt(x0.x * x0.x + x0.y * x0.y), nx = sqrt(nx2);
            const double2 ph = a0 > 0.0 ? make_double2(x0.x / a0, x0.y / a0) : make_double2(1.0, 0.0);
            alpha = make_double2(-ph.x * nx, -ph.y * nx);  // H x = alpha e_1
            const double2 v0 = make_double2(x0.x - alpha.x, x0.y - alpha.y);
            tau = 2.0 / (nx2 - a0 * a0 + (v0.x * v0.x + v0.y * v0.y));
            if (!(tau < 1e300)) tau = 0.0;
            __syncthreads();
            if (tid == 0 && tau != 0.0) x[k] = v0;
        }
        if (tid == 0) alph[k] = tau != 0.0 ? alpha : make_double2(0.0, 0.0);
        __syncthreads();
        if (tau != 0.0) hz_reflect<JT>(x, tau, k, K, A, K, k + 1, K);
        __syncthreads();
    }
    __syncthreads();
    for (int64_t e = tid; e < K * K; e += JT) {  // RH(c, r) = conj(R(r, c)); rows from kstop on are zero
        const int64_t r = e % K, c = e / K;
        const double2 v = r >= kstop ? make_double2(0.0, 0.0)
                                     : (r < c ? A[r + c * K] : (r == c ? alph[r] : make_double2(0.0, 0.0)));
        RH[c + r * K] = zconj(v);
    }
}

// dst[perm[i], q] = src[i, idx[q]] * sc[q]  (K x r; the rows go back through the pivoting)
__global__ void hz_select_perm_kernel(double2* dst, const double2* src, int64_t rows, const int32_t* idx,
                                      const double* sc, int64_t r, const int32_t* perm) {
    for (int64_t e = blockIdx.x * (int64_t)HT + threadIdx.x; e < rows * r; e += (int64_t)gridDim.x * HT) {
        const int64_t i = e % rows, q = e / rows;
        const double2 v = src[i + (int64_t)idx[q] * rows];
        dst[perm[i] + q * rows] = make_double2(v.x * sc[q], v.y * sc[q]);
    }
}

// FP32 arena chunks -> FP64 block buffers
struct GatherJob {
    int64_t src;      // arena offset (complex)
    double2* dst;     // block buffer
    int64_t ld_dst;
    int64_t r0, c0;   // position in the block
    int32_t ld_src, rows, ncols, pad_;
};
__global__ void hz_gather_kernel(const GatherJob* jobs, const float2* arena) {
    const GatherJob J = jobs[blockIdx.x];
    for (int64_t e = threadIdx.x; e < (int64_t)J.rows * J.ncols; e += HT) {
        const int64_t r = e % J.rows, c = e / J.rows;
        const float2 v = arena[J.src + r + c * J.ld_src];
        J.dst[(J.r0 + r) + (J.c0 + c) * J.ld_dst] = make_double2(v.x, v.y);
    }
}

__global__ void hz_perm_kernel(const int64_t* perm, const double2* in, double2* out, int64_t nc, int to_tree) {
    const int64_t q = blockIdx.x * (int64_t)HT + threadIdx.x;
    if (q >= 3 * nc) return;
    const int64_t p = q / 3, a = q - 3 * p, o = 3 * perm[p] + a;
    if (to_tree)
        out[q] = in[o];
    else
        out[o] = in[q];
}

// dst (cols x rows, ldd) = src^H (src rows x cols, lds)
__global__ void hz_adjoint_kernel(double2* dst, int64_t ldd, const double2* src, int64_t lds, int64_t rows,
                                  int64_t cols) {
    for (int64_t e = blockIdx.x * (int64_t)HT + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * HT) {
        const int64_t r = e % rows, c = e / rows;
        dst[c + r * ldd] = zconj(src[r + c * lds]);
    }
}

// Partial sums of |A_ij|^2 (rows x cols, lda), one per CTA
__global__ void __launch_bounds__(HT) hz_norm2_kernel(const double2* A, int64_t rows, int64_t cols, int64_t lda,
                                                      double* part) {
    __shared__ double red[HT / 32];
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)HT + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * HT) {
        const double2 v = A[e % rows + (e / rows) * lda];
        s += v.x * v.x + v.y * v.y;
    }
    s = hz_block_sum<HT>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// splitmix64 (Steele, Lea and Flood 2014): the counter-based source of the
// Gaussian test matrices of the randomized range finder
__device__ __forceinline__ uint64_t hz_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// O (n x l) with independent complex entries, real and imaginary parts N(0, 1)
// (Box-Muller on two uniforms in (0, 1] per entry)
__global__ void hz_gauss_kernel(double2* O, int64_t ne, uint64_t key) {
    for (int64_t e = blockIdx.x * (int64_t)HT + threadIdx.x; e < ne; e += (int64_t)gridDim.x * HT) {
        const uint64_t c = key * 0x100000000ull + 2 * (uint64_t)e;
        const double u1 = (double)((hz_splitmix64(c) >> 11) + 1) * 0x1.0p-53;
        const double u2 = (double)((hz_splitmix64(c + 1) >> 11) + 1) * 0x1.0p-53;
        const double r = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        O[e] = make_double2(r * cs, r * sn);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct HNode {
    int type = 0;  // 0 dense, 1 low rank, 2 subdivided
    int64_t m = 0, n = 0, k = 0, m0 = 0, n0 = 0;
    double2* D = nullptr;
    double2* U = nullptr;
    double2* V = nullptr;
    HNode* ch[4] = {nullptr, nullptr, nullptr, nullptr};
};

struct Ctx {
    cudaStream_t st;
    double eps;
    int* d_flag;  // zero pivot / Jacobi not converged
    int64_t launches = 0;
    uint64_t key = 0;  // test matrices drawn so far
    double* d_part = nullptr;  // hz_norm2_kernel partial sums
    int spawn = 0;     // nested forks still allowed (2^spawn chains at most)
    int device = 0;
};

// Runs f1 on C and f2 on a child context (its own stream and host thread)
// when C may still fork, else one after the other on C.  The two must touch
// disjoint blocks except for blocks both only read: the independent subtrees
// of the factorisation (the two triangular solves of an LU step, the column
// chains of a block triangular solve, the targets of a subdivided product).
// The child stream starts after everything issued on C so far, and C waits
// for the child before going on.
template <class F1, class F2>
void fork2(Ctx& C, F1&& f1, F2&& f2) {
    if (C.spawn <= 0) {
        f1(C);
        f2(C);
        return;
    }
    Ctx D{nullptr, C.eps, C.d_flag};
    D.key = C.key * 0x9e3779b97f4a7c15ull + 0x632be59bd9b4e019ull;  // a key space of its own
    D.device = C.device;
    const int sp = C.spawn;
    C.spawn = D.spawn = sp - 1;
    cudaEvent_t ev = nullptr;
    HM_CUDA(cudaStreamCreateWithFlags(&D.st, cudaStreamNonBlocking));
    HM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    HM_CUDA(cudaEventRecord(ev, C.st));
    HM_CUDA(cudaStreamWaitEvent(D.st, ev, 0));
    std::exception_ptr e1, e2;
    std::thread th([&] {
        try {
            HM_CUDA(cudaSetDevice(D.device));
            f2(D);
        } catch (...) {
            e2 = std::current_exception();
        }
    });
    try {
        f1(C);
    } catch (...) {
        e1 = std::current_exception();
    }
    th.join();
    C.spawn = sp;
    C.launches += D.launches;
    if (D.d_part) cudaFreeAsync(D.d_part, D.st);
    cudaEventRecord(ev, D.st);
    cudaStreamWaitEvent(C.st, ev, 0);
    if (e1 || e2) cudaStreamSynchronize(D.st);  // nothing of the child may still run on an error
    cudaEventDestroy(ev);
    cudaStreamDestroy(D.st);
    if (e1) std::rethrow_exception(e1);
    if (e2) std::rethrow_exception(e2);
}

double2* zalloc(Ctx& C, int64_t n) {
    double2* p = nullptr;
    HM_CUDA(cudaMallocAsync((void**)&p, (size_t)std::max<int64_t>(n, 1) * 16, C.st));
    return p;
}
void zfree(Ctx& C, double2* p) {
    if (p) HM_CUDA(cudaFreeAsync(p, C.st));
}
unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>(std::max<int64_t>(hm_cdiv(n, HT), 1), 4096); }

void gemm(Ctx& C, double2* c, const double2* a, const double2* b, int64_t M, int64_t N, int64_t K,
          int64_t lda, int64_t ldb, int64_t ldc, int opa, int opb, double2 alpha) {
    if (M <= 0 || N <= 0 || K <= 0) return;
    const int64_t tiles = hm_cdiv(M, TT) * hm_cdiv(N, TT);
    // few output tiles over a long contraction: split K over up to 2 CTAs per SM
    const int64_t splits = tiles >= 152 || K < 1024 ? 1 : std::min<int64_t>(hm_cdiv(K, 256), hm_cdiv(304, tiles));
    if (splits <= 1) {
        hz_gemm_kernel<<<(unsigned)tiles, HT, 0, C.st>>>(c, a, b, M, N, K, lda, ldb, ldc, opa, opb, alpha, K, 0);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
        C.launches++;
        return;
    }
    const int64_t kchunk = hm_cdiv(hm_cdiv(K, splits), TK) * TK;
    const int64_t sp = hm_cdiv(K, kchunk);
    double2* P = zalloc(C, sp * M * N);
    HM_CUDA(cudaMemsetAsync(P, 0, (size_t)sp * M * N * 16, C.st));
    hz_gemm_kernel<<<dim3((unsigned)tiles, (unsigned)sp), HT, 0, C.st>>>(P, a, b, M, N, K, lda, ldb, M, opa, opb,
                                                                          alpha, kchunk, M * N);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    hz_splitsum_kernel<<<grid_for(M * N), HT, 0, C.st>>>(c, ldc, P, M, N, sp);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    C.launches += 2;
    zfree(C, P);
}
void copy2d(Ctx& C, double2* dst, int64_t ldd, const double2* src, int64_t lds, int64_t rows, int64_t cols,
            double2 alpha, int add) {
    if (rows <= 0 || cols <= 0) return;
    hz_copy_kernel<<<grid_for(rows * cols), HT, 0, C.st>>>(dst, ldd, src, lds, rows, cols, alpha, add);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    C.launches++;
}
double2* identity(Ctx& C, int64_t n) {
    double2* p = zalloc(C, n * n);
    hz_identity_kernel<<<grid_for(n * n), HT, 0, C.st>>>(p, n);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    C.launches++;
    return p;
}
const double2 ONE = make_double2(1.0, 0.0), MONE = make_double2(-1.0, 0.0);

void free_tree(Ctx& C, HNode* x) {
    if (!x) return;
    for (HNode* c : x->ch) free_tree(C, c);
    zfree(C, x->D);
    zfree(C, x->U);
    zfree(C, x->V);
    delete x;
}

// Y (rows x c, ldy) += alpha op(x) X
void apply(Ctx& C, const HNode* x, int adj, const double2* X, int64_t ldx, double2* Y, int64_t ldy, int64_t c,
           double2 alpha) {
    if (c <= 0) return;
    if (x->type == 0) {
        gemm(C, Y, x->D, X, adj ? x->n : x->m, c, adj ? x->m : x->n, x->m, ldx, ldy, adj, 0, alpha);
    } else if (x->type == 1) {
        if (x->k == 0) return;
        const double2* A = adj ? x->U : x->V;  // contracted with X
        const double2* B = adj ? x->V : x->U;  // spans the result
        const int64_t la = adj ? x->m : x->n, lb = adj ? x->n : x->m;
        double2* T = zalloc(C, x->k * c);
        HM_CUDA(cudaMemsetAsync(T, 0, (size_t)x->k * c * 16, C.st));
        gemm(C, T, A, X, x->k, c, la, la, ldx, x->k, 1, 0, ONE);
        gemm(C, Y, B, T, lb, c, x->k, lb, x->k, ldy, 0, 0, alpha);
        zfree(C, T);
    } else {
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v) {
                const HNode* y = x->ch[2 * u + v];
                const int64_t ro = u ? x->m0 : 0, co = v ? x->n0 : 0;
                if (!adj)
                    apply(C, y, 0, X + co, ldx, Y + ro, ldy, c, alpha);
                else
                    apply(C, y, 1, X + ro, ldx, Y + co, ldy, c, alpha);
            }
    }
}

void trsm_leaf(Ctx& C, const HNode* x, double2* B, int64_t ldb, int64_t c, int mode) {
    if (c <= 0) return;
    const size_t smem = (size_t)TW * x->m * sizeof(double2);
    if (smem > 200 * 1024) hm_throw(HM_ERR_UNSUPPORTED, "H-LU: dense diagonal leaf above 3200 rows");
    if (smem > 48 * 1024)
        HM_CUDA(cudaFuncSetAttribute(hz_trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)std::min<int64_t>(hm_cdiv(c, TW), 4096);
    hz_trsm_kernel<<<grid, TW * 32, smem, C.st>>>(x->D, x->m, B, ldb, c, mode);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    C.launches++;
}
void solve_l(Ctx& C, const HNode* x, double2* B, int64_t ldb, int64_t c) {
    if (x->type == 0) return trsm_leaf(C, x, B, ldb, c, 0);
    solve_l(C, x->ch[0], B, ldb, c);
    apply(C, x->ch[2], 0, B, ldb, B + x->m0, ldb, c, MONE);
    solve_l(C, x->ch[3], B + x->m0, ldb, c);
}
void solve_u(Ctx& C, const HNode* x, double2* B, int64_t ldb, int64_t c) {
    if (x->type == 0) return trsm_leaf(C, x, B, ldb, c, 1);
    solve_u(C, x->ch[3], B + x->m0, ldb, c);
    apply(C, x->ch[1], 0, B + x->m0, ldb, B, ldb, c, MONE);
    solve_u(C, x->ch[0], B, ldb, c);
}
void solve_uh(Ctx& C, const HNode* x, double2* B, int64_t ldb, int64_t c) {
    if (x->type == 0) return trsm_leaf(C, x, B, ldb, c, 2);
    solve_uh(C, x->ch[0], B, ldb, c);
    apply(C, x->ch[1], 1, B, ldb, B + x->n0, ldb, c, MONE);
    solve_uh(C, x->ch[3], B + x->n0, ldb, c);
}

// dst (cols x rows, ldd) = src^H
void adjoint(Ctx& C, double2* dst, int64_t ldd, const double2* src, int64_t lds, int64_t rows, int64_t cols) {
    if (rows <= 0 || cols <= 0) return;
    hz_adjoint_kernel<<<grid_for(rows * cols), HT, 0, C.st>>>(dst, ldd, src, lds, rows, cols);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    C.launches++;
}

constexpr int NORM_CTAS = 128;

// ||A||_F^2 (rows x cols, lda); synchronises the stream
double norm2(Ctx& C, const double2* A, int64_t rows, int64_t cols, int64_t lda) {
    if (rows <= 0 || cols <= 0) return 0.0;
    if (!C.d_part) HM_CUDA(cudaMallocAsync((void**)&C.d_part, NORM_CTAS * sizeof(double), C.st));
    hz_norm2_kernel<<<NORM_CTAS, HT, 0, C.st>>>(A, rows, cols, lda, C.d_part);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    C.launches++;
    double part[NORM_CTAS];
    HM_CUDA(cudaMemcpyAsync(part, C.d_part, sizeof(part), cudaMemcpyDeviceToHost, C.st));
    HM_CUDA(cudaStreamSynchronize(C.st));
    double s = 0.0;
    for (int i = 0; i < NORM_CTAS; ++i) s += part[i];
    return s;
}

// D (x->m x x->n, ldd) += alpha x, the node written out densely
void densify(Ctx& C, const HNode* x, double2* D, int64_t ldd, double2 alpha) {
    if (x->type == 0) return copy2d(C, D, ldd, x->D, x->m, x->m, x->n, alpha, 1);
    if (x->type == 1) return gemm(C, D, x->U, x->V, x->m, x->n, x->k, x->m, x->n, ldd, 0, 1, alpha);
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v)
            densify(C, x->ch[2 * u + v], D + (u ? x->m0 : 0) + (v ? x->n0 : 0) * ldd, ldd, alpha);
}

// Recompression (Sec. 3.2) of U2 V2^H (m x K, n x K; both freed) into x->U,
// x->V, x->k: QR of both factors, SVD of R_U R_V^H, the smallest rank r whose
// discarded singular values, together with an error rho2 already committed
// (squared Frobenius norm), stay within eps_LU of the whole.
// One-sided Jacobi of W (K x K) -> WJ = P S, s: a cluster of CJ CTAs for K up
// to CJ_MAX, else one CTA on global memory.  Rotations stop at max(K u, 1e-15)
// of orthogonality: the Gram form divides by the singular values it keeps
// (P_r = W L_r S_r^-1), so a looser stop would be amplified by up to 1/eps_LU.
void jacobi(Ctx& C, const double2* W, double2* WJ, int64_t K, double* s) {
    const double tol_min = 1e-15;
    if (K <= CJ_MAX) {
        const size_t sm = (size_t)4 * ((K + NBJ - 1) / NBJ) * K * sizeof(double2);
        hz_jacobi_cluster_kernel<<<CJ, CJT, sm, C.st>>>(W, WJ, K, s, C.d_flag, tol_min);
    } else {
        hz_jacobi_kernel<<<1, JT, 0, C.st>>>(W, WJ, K, s, C.d_flag, tol_min);
    }
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    C.launches++;
}

// SVD of the recompression core W (K x K) = P S L^H: the one-sided Jacobi runs
// on R^H of the pivoted QR W Pi = Q R, whose columns converge to X S with
// R^H = X S Y^H, so L = Pi X (for K above QP_MAX: on W^H, L = X).  Ranks by the
// truncation rule with rho2 already spent; ord sorts the singular values.
struct CoreSvd {
    double2* XS = nullptr;  // K x K, columns X_j s_j
    int32_t* perm = nullptr;
    std::vector<double> hs;
    std::vector<int32_t> ord;
    int64_t r = 0;
};

void core_svd(Ctx& C, const double2* W, int64_t K, double rho2, CoreSvd& out) {
    double2* RH = zalloc(C, K * K);
    HM_CUDA(cudaMallocAsync((void**)&out.perm, (size_t)K * 4, C.st));
    if (K <= QP_MAX) {
        const size_t sm = K <= QP_SMEM ? (size_t)K * K * sizeof(double2) : 0;
        double2* A = K <= QP_SMEM ? nullptr : zalloc(C, K * K);
        hz_qrcp_kernel<<<1, JT, sm, C.st>>>(W, A, RH, out.perm, K);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
        C.launches++;
        zfree(C, A);
    } else {
        adjoint(C, RH, K, W, K, K, K);
        std::vector<int32_t> id(K);
        for (int64_t i = 0; i < K; ++i) id[i] = (int32_t)i;
        HM_CUDA(cudaMemcpyAsync(out.perm, id.data(), (size_t)K * 4, cudaMemcpyHostToDevice, C.st));
        HM_CUDA(cudaStreamSynchronize(C.st));
    }
    out.XS = zalloc(C, K * K);
    double* s = nullptr;
    HM_CUDA(cudaMallocAsync((void**)&s, (size_t)K * 8, C.st));
    jacobi(C, RH, out.XS, K, s);
    out.hs.assign(K, 0.0);
    HM_CUDA(cudaMemcpyAsync(out.hs.data(), s, (size_t)K * 8, cudaMemcpyDeviceToHost, C.st));
    HM_CUDA(cudaStreamSynchronize(C.st));
    HM_CUDA(cudaFreeAsync(s, C.st));
    zfree(C, RH);
    const std::vector<double>& hs = out.hs;
    for (int64_t i = 0; i < K; ++i)
        if (!std::isfinite(hs[i])) hm_throw(HM_ERR_NUMERIC, "H-LU: non-finite singular value");
    out.ord.resize(K);
    for (int64_t i = 0; i < K; ++i) out.ord[i] = (int32_t)i;
    std::stable_sort(out.ord.begin(), out.ord.end(), [&](int32_t a, int32_t b) { return hs[a] > hs[b]; });
    double tot = rho2;
    for (int64_t i = 0; i < K; ++i) tot += hs[i] * hs[i];
    int64_t r = K;
    double tail = rho2;
    for (int64_t i = K - 1; i >= 0; --i) {
        const double sv = hs[out.ord[i]];
        if (std::sqrt(tail + sv * sv) <= C.eps * std::sqrt(tot)) {
            tail += sv * sv;
            r = i;
        } else {
            break;
        }
    }
    while (r > 0 && !(hs[out.ord[r - 1]] > 0.0)) --r;
    out.r = r;
}

void core_free(Ctx& C, CoreSvd& cs) {
    zfree(C, cs.XS);
    if (cs.perm) HM_CUDA(cudaFreeAsync(cs.perm, C.st));
    cs.XS = nullptr;
    cs.perm = nullptr;
}

// L_r S_r^e (K x r) from the core's X S: column q is (X S)_ord[q] s_ord[q]^(e - 1),
// its rows put back through Pi
double2* l_scaled(Ctx& C, const CoreSvd& cs, int64_t K, double e) {
    const int64_t r = cs.r;
    std::vector<double> sc(r);
    for (int64_t q = 0; q < r; ++q) sc[q] = std::pow(cs.hs[cs.ord[q]], e - 1.0);
    int32_t* d_ord = nullptr;
    double* d_sc = nullptr;
    HM_CUDA(cudaMallocAsync((void**)&d_ord, (size_t)r * 4, C.st));
    HM_CUDA(cudaMallocAsync((void**)&d_sc, (size_t)r * 8, C.st));
    HM_CUDA(cudaMemcpyAsync(d_ord, cs.ord.data(), (size_t)r * 4, cudaMemcpyHostToDevice, C.st));
    HM_CUDA(cudaMemcpyAsync(d_sc, sc.data(), (size_t)r * 8, cudaMemcpyHostToDevice, C.st));
    double2* L = zalloc(C, K * r);
    hz_select_perm_kernel<<<grid_for(K * r), HT, 0, C.st>>>(L, cs.XS, K, d_ord, d_sc, r, cs.perm);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    C.launches++;
    HM_CUDA(cudaFreeAsync(d_ord, C.st));
    HM_CUDA(cudaFreeAsync(d_sc, C.st));
    return L;
}

// eps_LU from which the Gram form below replaces the Householder QR
constexpr double GRAM_EPS = 1e-5;
void truncate_gram(Ctx& C, HNode* x, double2* U2, double2* V2, int64_t K, double rho2);

void truncate(Ctx& C, HNode* x, double2* U2, double2* V2, int64_t K, double rho2 = 0.0) {
    if (C.eps >= GRAM_EPS && K <= JS_MAX_CHOL) return truncate_gram(C, x, U2, V2, K, rho2);
    const int64_t m = x->m, n = x->n;
    double2 *QU = zalloc(C, m * K), *RU = zalloc(C, K * K), *QV = zalloc(C, n * K), *RV = zalloc(C, K * K);
    const size_t smem = (size_t)K * sizeof(double);
    if (smem > 48 * 1024)
        HM_CUDA(cudaFuncSetAttribute(hz_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    hz_qr_kernel<<<1, QT, smem, C.st>>>(U2, m, K, QU, RU);
    HM_LAUNCHED();
    hz_qr_kernel<<<1, QT, smem, C.st>>>(V2, n, K, QV, RV);
    HM_LAUNCHED();
    HM_CUDA(cudaGetLastError());
    C.launches += 2;
    zfree(C, U2);
    zfree(C, V2);
    double2* W = zalloc(C, K * K);
    HM_CUDA(cudaMemsetAsync(W, 0, (size_t)K * K * 16, C.st));
    gemm(C, W, RU, RV, K, K, K, K, K, K, 0, 1, ONE);  // R_U R_V^H
    CoreSvd cs;
    core_svd(C, W, K, rho2, cs);
    zfree(C, x->U);
    zfree(C, x->V);
    x->U = x->V = nullptr;
    const int64_t r = cs.r;
    x->k = r;
    if (r > 0) {
        // U = Q_U P_r S_r^{1/2} = Q_U W L_r S_r^{-1/2},  V = Q_V L_r S_r^{1/2}
        double2* Lh = l_scaled(C, cs, K, 0.5);
        double2* Lm = l_scaled(C, cs, K, -0.5);
        double2* WL = zalloc(C, K * r);
        HM_CUDA(cudaMemsetAsync(WL, 0, (size_t)K * r * 16, C.st));
        gemm(C, WL, W, Lm, K, r, K, K, K, K, 0, 0, ONE);
        x->U = zalloc(C, m * r);
        x->V = zalloc(C, n * r);
        HM_CUDA(cudaMemsetAsync(x->U, 0, (size_t)m * r * 16, C.st));
        HM_CUDA(cudaMemsetAsync(x->V, 0, (size_t)n * r * 16, C.st));
        gemm(C, x->U, QU, WL, m, r, K, m, K, m, 0, 0, ONE);
        gemm(C, x->V, QV, Lh, n, r, K, n, K, n, 0, 0, ONE);
        zfree(C, Lh);
        zfree(C, Lm);
        zfree(C, WL);
    }
    core_free(C, cs);
    zfree(C, W);
    zfree(C, QU);
    zfree(C, RU);
    zfree(C, QV);
    zfree(C, RV);
}

// The same recompression in Gram form, for eps_LU >= GRAM_EPS: R_U, R_V from
// the Cholesky factors of U2^H U2 and V2^H V2 (split-K GEMMs over the long
// side, many CTAs), and the orthonormal factors never formed: with
// W = R_U R_V^H = P S L^H,
//   Q_U P_r S_r^{1/2} = U2 T_U,  T_U = R_V^H L_r S_r^{-1/2},
//   Q_V L_r S_r^{1/2} = V2 T_V,  T_V = R_U^H P_r S_r^{-1/2},
// valid for singular R_U, R_V; L_r S_r = W^H P_r.  The Gram matrices square
// the conditioning: directions below 3.2e-7 of a column are dropped, hence
// the eps_LU floor (30 times that level).

void truncate_gram(Ctx& C, HNode* x, double2* U2, double2* V2, int64_t K, double rho2) {
    const int64_t m = x->m, n = x->n;
    double2 *GU = zalloc(C, K * K), *GV = zalloc(C, K * K);
    HM_CUDA(cudaMemsetAsync(GU, 0, (size_t)K * K * 16, C.st));
    HM_CUDA(cudaMemsetAsync(GV, 0, (size_t)K * K * 16, C.st));
    gemm(C, GU, U2, U2, K, K, m, m, m, K, 1, 0, ONE);
    gemm(C, GV, V2, V2, K, K, n, n, n, K, 1, 0, ONE);
    double2* W = zalloc(C, K * K);
    const size_t gsm = K <= QP_SMEM ? (size_t)K * K * sizeof(double2) : 0;
    hz_gram_core_kernel<<<1, JT, gsm, C.st>>>(GU, GV, W, K);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    C.launches++;
    CoreSvd cs;
    core_svd(C, W, K, rho2, cs);
    zfree(C, x->U);
    zfree(C, x->V);
    x->U = x->V = nullptr;
    const int64_t r = cs.r;
    x->k = r;
    if (r > 0) {
        double2* Lm = l_scaled(C, cs, K, -0.5);   // L_r S_r^{-1/2}
        double2* Lm3 = l_scaled(C, cs, K, -1.5);  // L_r S_r^{-3/2}
        double2 *WL = zalloc(C, K * r), *TU = zalloc(C, K * r), *TV = zalloc(C, K * r);
        HM_CUDA(cudaMemsetAsync(WL, 0, (size_t)K * r * 16, C.st));
        HM_CUDA(cudaMemsetAsync(TU, 0, (size_t)K * r * 16, C.st));
        HM_CUDA(cudaMemsetAsync(TV, 0, (size_t)K * r * 16, C.st));
        gemm(C, WL, W, Lm3, K, r, K, K, K, K, 0, 0, ONE);  // W L_r S^{-3/2} = P_r S^{-1/2}
        gemm(C, TU, GV, Lm, K, r, K, K, K, K, 1, 0, ONE);  // R_V^H L_r S^{-1/2}
        gemm(C, TV, GU, WL, K, r, K, K, K, K, 1, 0, ONE);  // R_U^H P_r S^{-1/2}
        x->U = zalloc(C, m * r);
        x->V = zalloc(C, n * r);
        HM_CUDA(cudaMemsetAsync(x->U, 0, (size_t)m * r * 16, C.st));
        HM_CUDA(cudaMemsetAsync(x->V, 0, (size_t)n * r * 16, C.st));
        gemm(C, x->U, U2, TU, m, r, K, m, K, m, 0, 0, ONE);
        gemm(C, x->V, V2, TV, n, r, K, n, K, n, 0, 0, ONE);
        zfree(C, Lm);
        zfree(C, Lm3);
        zfree(C, WL);
        zfree(C, TU);
        zfree(C, TV);
    }
    core_free(C, cs);
    zfree(C, U2);
    zfree(C, V2);
    zfree(C, GU);
    zfree(C, GV);
    zfree(C, W);
}

// Largest side up to which a dense matrix is recompressed exactly (QR of D, or
// of D^H, and the SVD of its triangle); larger ones go through the range finder.
constexpr int64_t EXACT_SIDE = 63;

// x (low rank) <- the eps_LU truncation of the dense D (m x n; freed).  Small
// blocks: exact, as the low-rank sum D I^H (or I D^H).  Larger blocks: an
// adaptive randomized range finder (Halko, Martinsson and Tropp 2011): Q =
// orth(D Omega) with l = 32, 64, ... Gaussian columns until the residual
// ||D - Q Q^H D||_F, computed exactly, is at most eps_LU ||D||_F / 2; then the
// recompression of Q (D^H Q)^H with that residual counted in its tail.  Where
// l would pass half the smaller side, the exact path.
void compress_dense(Ctx& C, HNode* x, double2* D) {
    const int64_t m = x->m, n = x->n, mn = std::min(m, n);
    if (mn > EXACT_SIDE) {
        const double d2 = norm2(C, D, m, n, m);
        if (d2 == 0.0) {
            zfree(C, D);
            zfree(C, x->U);
            zfree(C, x->V);
            x->U = x->V = nullptr;
            x->k = 0;
            return;
        }
        for (int64_t l = 32; 2 * l <= mn; l *= 2) {
            double2* O = zalloc(C, n * l);
            hz_gauss_kernel<<<grid_for(n * l), HT, 0, C.st>>>(O, n * l, ++C.key);
            HM_CUDA(cudaGetLastError());
            HM_LAUNCHED();
            C.launches++;
            double2* Y = zalloc(C, m * l);
            HM_CUDA(cudaMemsetAsync(Y, 0, (size_t)m * l * 16, C.st));
            gemm(C, Y, D, O, m, l, n, m, n, m, 0, 0, ONE);  // D Omega
            zfree(C, O);
            double2 *Q = zalloc(C, m * l), *R = zalloc(C, l * l);
            hz_qr_kernel<<<1, QT, (size_t)l * sizeof(double), C.st>>>(Y, m, l, Q, R);
            HM_CUDA(cudaGetLastError());
            HM_LAUNCHED();
            C.launches++;
            zfree(C, Y);
            zfree(C, R);
            double2* V2 = zalloc(C, n * l);
            HM_CUDA(cudaMemsetAsync(V2, 0, (size_t)n * l * 16, C.st));
            gemm(C, V2, D, Q, n, l, m, m, m, n, 1, 0, ONE);  // D^H Q
            double2* E = zalloc(C, m * n);
            copy2d(C, E, m, D, m, m, n, ONE, 0);
            gemm(C, E, Q, V2, m, n, l, m, n, m, 0, 1, MONE);  // D - Q Q^H D
            const double rho2 = norm2(C, E, m, n, m);
            zfree(C, E);
            if (rho2 <= 0.25 * C.eps * C.eps * d2) {
                zfree(C, D);
                truncate(C, x, Q, V2, l, rho2);
                return;
            }
            zfree(C, Q);
            zfree(C, V2);
        }
    }
    double2 *U2, *V2;
    if (m >= n) {
        U2 = D;
        V2 = identity(C, n);
    } else {
        U2 = identity(C, m);
        V2 = zalloc(C, n * m);
        adjoint(C, V2, n, D, m, m, n);
        zfree(C, D);
    }
    truncate(C, x, U2, V2, mn);
}

// x += alpha Up Vp^H
void add_lr(Ctx& C, HNode* x, const double2* Up, int64_t lu, const double2* Vp, int64_t lv, int64_t k,
            double2 alpha) {
    if (k <= 0) return;
    if (x->type == 0) {
        gemm(C, x->D, Up, Vp, x->m, x->n, k, lu, lv, x->m, 0, 1, alpha);
        return;
    }
    if (x->type == 2) {
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v)
                add_lr(C, x->ch[2 * u + v], Up + (u ? x->m0 : 0), lu, Vp + (v ? x->n0 : 0), lv, k, alpha);
        return;
    }
    const int64_t K = x->k + k, m = x->m, n = x->n;
    if (K > std::min(m, n)) {  // the sum densely
        double2* D = zalloc(C, m * n);
        HM_CUDA(cudaMemsetAsync(D, 0, (size_t)m * n * 16, C.st));
        densify(C, x, D, m, ONE);
        gemm(C, D, Up, Vp, m, n, k, lu, lv, m, 0, 1, alpha);
        return compress_dense(C, x, D);
    }
    double2* U2 = zalloc(C, m * K);
    double2* V2 = zalloc(C, n * K);
    if (x->k) {
        copy2d(C, U2, m, x->U, m, m, x->k, ONE, 0);
        copy2d(C, V2, n, x->V, n, n, x->k, ONE, 0);
    }
    copy2d(C, U2 + m * x->k, m, Up, lu, m, k, alpha, 0);
    copy2d(C, V2 + n * x->k, n, Vp, lv, n, k, ONE, 0);
    truncate(C, x, U2, V2, K);
}

// x += alpha P (m x n, ld lp)
void add_dense(Ctx& C, HNode* x, const double2* P, int64_t lp, double2 alpha) {
    if (x->type == 0) return copy2d(C, x->D, x->m, P, lp, x->m, x->n, alpha, 1);
    if (x->type == 2) {
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v)
                add_dense(C, x->ch[2 * u + v], P + (u ? x->m0 : 0) + (v ? x->n0 : 0) * lp, lp, alpha);
        return;
    }
    double2* D = zalloc(C, x->m * x->n);
    HM_CUDA(cudaMemsetAsync(D, 0, (size_t)x->m * x->n * 16, C.st));
    densify(C, x, D, x->m, ONE);
    copy2d(C, D, x->m, P, lp, x->m, x->n, alpha, 1);
    compress_dense(C, x, D);
}

// C -= A B
void gemm_sub(Ctx& C, HNode* c, const HNode* a, const HNode* b) {
    if (c->type == 2 && a->type == 2 && b->type == 2) {  // four independent targets
        auto target = [&](Ctx& X, int u, int v) {
            for (int w = 0; w < 2; ++w) gemm_sub(X, c->ch[2 * u + v], a->ch[2 * u + w], b->ch[2 * w + v]);
        };
        auto row = [&](Ctx& X, int u) {
            fork2(X, [&](Ctx& Y) { target(Y, u, 0); }, [&](Ctx& Y) { target(Y, u, 1); });
        };
        fork2(C, [&](Ctx& X) { row(X, 0); }, [&](Ctx& X) { row(X, 1); });
        return;
    }
    if (b->type == 1) {  // A (U_b V_b^H) = (A U_b) V_b^H
        if (b->k == 0) return;
        double2* AU = zalloc(C, a->m * b->k);
        HM_CUDA(cudaMemsetAsync(AU, 0, (size_t)a->m * b->k * 16, C.st));
        apply(C, a, 0, b->U, b->m, AU, a->m, b->k, ONE);
        add_lr(C, c, AU, a->m, b->V, b->n, b->k, MONE);
        zfree(C, AU);
        return;
    }
    if (a->type == 1) {  // (U_a V_a^H) B = U_a (B^H V_a)^H
        if (a->k == 0) return;
        double2* BV = zalloc(C, b->n * a->k);
        HM_CUDA(cudaMemsetAsync(BV, 0, (size_t)b->n * a->k * 16, C.st));
        apply(C, b, 1, a->V, a->n, BV, b->n, a->k, ONE);
        add_lr(C, c, a->U, a->m, BV, b->n, a->k, MONE);
        zfree(C, BV);
        return;
    }
    // dense or subdivided operands: A times B written out densely
    double2* Bd = zalloc(C, b->m * b->n);
    HM_CUDA(cudaMemsetAsync(Bd, 0, (size_t)b->m * b->n * 16, C.st));
    densify(C, b, Bd, b->m, ONE);
    if (c->type == 0) {
        apply(C, a, 0, Bd, b->m, c->D, c->m, b->n, MONE);
        zfree(C, Bd);
        return;
    }
    double2* P = zalloc(C, a->m * b->n);
    HM_CUDA(cudaMemsetAsync(P, 0, (size_t)a->m * b->n * 16, C.st));
    apply(C, a, 0, Bd, b->m, P, a->m, b->n, ONE);
    zfree(C, Bd);
    add_dense(C, c, P, a->m, MONE);
    zfree(C, P);
}

void trsm_l(Ctx& C, const HNode* L, HNode* X) {
    if (X->type == 0) return solve_l(C, L, X->D, X->m, X->n);
    if (X->type == 1) return solve_l(C, L, X->U, X->m, X->k);
    auto column = [&](Ctx& Y, int v) {  // the two block columns are independent
        trsm_l(Y, L->ch[0], X->ch[v]);
        gemm_sub(Y, X->ch[2 + v], L->ch[2], X->ch[v]);
        trsm_l(Y, L->ch[3], X->ch[2 + v]);
    };
    fork2(C, [&](Ctx& Y) { column(Y, 0); }, [&](Ctx& Y) { column(Y, 1); });
}

void trsm_u(Ctx& C, const HNode* U, HNode* X) {
    if (X->type == 0) {  // X^H <- U^{-H} X^H
        double2* T = zalloc(C, X->m * X->n);
        adjoint(C, T, X->n, X->D, X->m, X->m, X->n);
        solve_uh(C, U, T, X->n, X->m);
        adjoint(C, X->D, X->m, T, X->n, X->n, X->m);
        zfree(C, T);
        return;
    }
    if (X->type == 1) return solve_uh(C, U, X->V, X->n, X->k);
    auto row = [&](Ctx& Y, int u) {  // the two block rows are independent
        trsm_u(Y, U->ch[0], X->ch[2 * u]);
        gemm_sub(Y, X->ch[2 * u + 1], X->ch[2 * u], U->ch[1]);
        trsm_u(Y, U->ch[3], X->ch[2 * u + 1]);
    };
    fork2(C, [&](Ctx& Y) { row(Y, 0); }, [&](Ctx& Y) { row(Y, 1); });
}

void lu(Ctx& C, HNode* x) {
    if (x->type == 0) {
        hz_getrf_kernel<<<1, HT, 0, C.st>>>(x->D, x->m, C.d_flag);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
        C.launches++;
        return;
    }
    lu(C, x->ch[0]);                        // 1. A11 = L11 U11
    fork2(C, [&](Ctx& Y) { trsm_l(Y, x->ch[0], x->ch[1]); },   // 2. U12 = L11^{-1} A12
          [&](Ctx& Y) { trsm_u(Y, x->ch[0], x->ch[2]); });     // 3. L21 = A21 U11^{-1}
    gemm_sub(C, x->ch[3], x->ch[2], x->ch[1]);  // 4. A22 - L21 U12 ...
    lu(C, x->ch[3]);                        //    = L22 U22
}

int64_t stored(const HNode* x) {
    if (x->type == 0) return x->m * x->n;
    if (x->type == 1) return (x->m + x->n) * x->k;
    int64_t s = 0;
    for (const HNode* c : x->ch) s += stored(c);
    return s;
}

struct Hlu {
    HNode* root = nullptr;
    double eps = 0;
    double seconds = 0;
    int64_t launches = 0;
};

}  // namespace

// Builds the block tree from the handle's partition and its stored factors
// (FP32 arena -> FP64), factorises it, and keeps it in the handle.
void hlu_factor(hm_matrix* h, double eps_lu, cudaStream_t st) {
    hlu_release(h, st);
    const auto t0 = std::chrono::steady_clock::now();
    Ctx C{st, eps_lu, nullptr, 0};
    C.spawn = 4;  // up to 16 independent chains in flight
    HM_CUDA(cudaGetDevice(&C.device));
    // shared-memory limits of the core kernels, set once before any chain forks
    HM_CUDA(cudaFuncSetAttribute(hz_jacobi_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(4 * ((CJ_MAX + NBJ - 1) / NBJ) * CJ_MAX * sizeof(double2))));
    HM_CUDA(cudaFuncSetAttribute(hz_qrcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(QP_SMEM * QP_SMEM * sizeof(double2))));
    HM_CUDA(cudaFuncSetAttribute(hz_gram_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(QP_SMEM * QP_SMEM * sizeof(double2))));
    HM_CUDA(cudaMallocAsync((void**)&C.d_flag, sizeof(int), st));
    HM_CUDA(cudaMemsetAsync(C.d_flag, 0, sizeof(int), st));
    std::map<std::pair<int64_t, int64_t>, int64_t> bmap;
    for (int64_t b = 0; b < (int64_t)h->blocks.size(); ++b) bmap[{h->blocks[b].tau, h->blocks[b].sigma}] = b;
    std::vector<HNode*> leaf_of(h->blocks.size(), nullptr);
    HNode* root = nullptr;
    try {
        std::function<HNode*(int64_t, int64_t)> build = [&](int64_t t, int64_t s) -> HNode* {
            const hm_cluster& ct = h->clusters[t];
            const hm_cluster& cs = h->clusters[s];
            HNode* x = new HNode();
            x->m = 3 * (ct.end - ct.begin);
            x->n = 3 * (cs.end - cs.begin);
            auto it = bmap.find({t, s});
            if (it != bmap.end()) {
                const hm_block& B = h->blocks[it->second];
                leaf_of[it->second] = x;
                if (B.admissible) {
                    x->type = 1;
                    x->k = B.rank;
                    x->U = zalloc(C, x->m * x->k);
                    x->V = zalloc(C, x->n * x->k);
                } else {
                    x->type = 0;
                    x->D = zalloc(C, x->m * x->n);
                }
                return x;
            }
            if (ct.is_leaf || cs.is_leaf) hm_throw(HM_ERR_CUDA, "H-LU: block tree and partition disagree");
            x->type = 2;
            const int64_t tc[2] = {ct.child0, ct.child1}, sc[2] = {cs.child0, cs.child1};
            for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v) x->ch[2 * u + v] = build(tc[u], sc[v]);
            x->m0 = x->ch[0]->m;
            x->n0 = x->ch[0]->n;
            return x;
        };
        root = build(0, 0);
        // the stored chunks into the FP64 blocks
        std::vector<GatherJob> jobs;
        for (const Chunk& c : h->plan.chunks) {
            if (c.ncols == 0) continue;
            HNode* x = leaf_of[c.block];
            const hm_block& B = h->blocks[c.block];
            const hm_cluster& t = h->clusters[B.tau];
            const hm_cluster& s = h->clusters[B.sigma];
            GatherJob J;
            J.src = c.data;
            J.ld_src = c.ld;
            J.rows = c.rows;
            J.ncols = c.ncols;
            J.pad_ = 0;
            if (c.kind == 2) {
                J.dst = x->V;
                J.ld_dst = x->n;
                J.r0 = c.leaf_dof - 3 * s.begin;
                J.c0 = 0;
            } else {
                J.dst = c.kind == 1 ? x->U : x->D;
                J.ld_dst = x->m;
                J.r0 = c.leaf_dof - 3 * t.begin;
                J.c0 = c.kind == 0 ? c.vec - 3 * s.begin : 0;
            }
            jobs.push_back(J);
        }
        if (!jobs.empty()) {
            GatherJob* d = nullptr;
            HM_CUDA(cudaMallocAsync((void**)&d, jobs.size() * sizeof(GatherJob), st));
            HM_CUDA(cudaMemcpyAsync(d, jobs.data(), jobs.size() * sizeof(GatherJob), cudaMemcpyHostToDevice, st));
            hz_gather_kernel<<<(unsigned)jobs.size(), HT, 0, st>>>(d, (const float2*)matvec_arena(h->mv));
            HM_CUDA(cudaGetLastError());
            HM_LAUNCHED();
            HM_CUDA(cudaFreeAsync(d, st));
        }
        lu(C, root);
        int flag = 0;
        HM_CUDA(cudaMemcpyAsync(&flag, C.d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        if (flag & 1) hm_throw(HM_ERR_NUMERIC, "H-LU: zero pivot in a dense diagonal leaf");
        if (flag & 2) hm_throw(HM_ERR_NUMERIC, "H-LU: one-sided Jacobi not converged in 80 sweeps");
    } catch (...) {
        cudaStreamSynchronize(st);
        free_tree(C, root);
        cudaFree(C.d_flag);
        if (C.d_part) cudaFree(C.d_part);
        throw;
    }
    HM_CUDA(cudaFreeAsync(C.d_flag, st));
    if (C.d_part) HM_CUDA(cudaFreeAsync(C.d_part, st));
    HM_CUDA(cudaStreamSynchronize(st));
    Hlu* F = new Hlu();
    F->root = root;
    F->eps = eps_lu;
    F->launches = C.launches;
    F->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    h->hlu = F;
}

void hlu_solve(hm_matrix* h, int32_t nrhs, const double2* b, double2* x, cudaStream_t st) {
    Hlu* F = (Hlu*)h->hlu;
    if (!F) hm_throw(HM_ERR_ARG, "no H-LU factors: call hm_lu_factor first");
    Ctx C{st, F->eps, nullptr, 0};
    const int64_t N = 3 * h->nc;
    double2* y = zalloc(C, N * nrhs);
    for (int32_t j = 0; j < nrhs; ++j) {
        hz_perm_kernel<<<(unsigned)hm_cdiv(N, HT), HT, 0, st>>>(h->d_perm, b + j * N, y + j * N, h->nc, 1);
        HM_LAUNCHED();
    }
    HM_CUDA(cudaGetLastError());
    solve_l(C, F->root, y, N, nrhs);
    solve_u(C, F->root, y, N, nrhs);
    for (int32_t j = 0; j < nrhs; ++j) {
        hz_perm_kernel<<<(unsigned)hm_cdiv(N, HT), HT, 0, st>>>(h->d_perm, y + j * N, x + j * N, h->nc, 0);
        HM_LAUNCHED();
    }
    HM_CUDA(cudaGetLastError());
    zfree(C, y);
}

void hlu_info(const hm_matrix* h, double* seconds, int64_t* entries, int64_t* launches) {
    const Hlu* F = (const Hlu*)h->hlu;
    if (!F) hm_throw(HM_ERR_ARG, "no H-LU factors");
    if (seconds) *seconds = F->seconds;
    if (entries) *entries = stored(F->root);
    if (launches) *launches = F->launches;
}

void hlu_release(hm_matrix* h, cudaStream_t st) {
    Hlu* F = (Hlu*)h->hlu;
    if (!F) return;
    Ctx C{st, 0, nullptr, 0};
    free_tree(C, F->root);
    cudaStreamSynchronize(st);
    delete F;
    h->hlu = nullptr;
}

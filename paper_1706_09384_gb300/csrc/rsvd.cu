// rsvd.cu — randomized SVD for the admissible blocks whose rows the vector ACA
// cannot pivot (the remark closing Sec. 2.3: for configurations where every
// 3x3 sub-block of the double-layer kernel T is singular, the randomized SVD
// of Liberty, Woolfe, Martinsson, Rokhlin & Tygert (2007) is preferred).
//
// For a block A (3m x 3n), l samples:
//   1. Omega (3n x (l + p)): complex normal entries, E|w|^2 = 1, by the
//      Box-Muller transform of two uniforms from splitmix64 (Steele, Lea &
//      Flood 2014) of the counter j * 1024 + c under a key made from the
//      block's first row and column point (tree order of its own problem);
//   2. Y = A Omega;
//   3. Householder QR of Y's first l columns, applied to the p probe columns
//      as well: the probes' entries below row l are then (I - Q Q^H) A w, and
//      the mean of their squared norms estimates ||(I - Q Q^H) A||_F^2;
//   4. accepted when that mean is at most (eps/4)^2 ||A||_F^2, else l doubles
//      (up to min(3m, 3n, 768));
//   5. Q formed explicitly, V = A^H Q, so A ~ Q V^H; the factors then go
//      through the recompression of Sec. 3.2 with eps sqrt(3)/2 (the range
//      and truncation errors are orthogonal: total <= eps ||A||_F).
// A, Y, Omega, Q and V are FP64 (the block is evaluated once, in FP64, like
// the ACA's rows and columns); one CTA runs the QR of one block.
#include <algorithm>
#include <cmath>
#include <vector>

#include "green.cuh"
#include "hm_internal.h"

namespace {

constexpr int RS_L0 = 64;
constexpr int RS_P = 8;
constexpr int RS_LMAX = 768;
constexpr uint64_t RS_CSTRIDE = 1024;
constexpr int RS_THREADS = 256;
constexpr int GT = 32;  // GEMM tile (rows and columns)
constexpr int GK = 16;  // GEMM K step

HM_HD uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ double2 rs_gauss(uint64_t key, uint64_t ctr) {
    const uint64_t a = splitmix64(key ^ splitmix64(2 * ctr));
    const uint64_t b = splitmix64(key ^ splitmix64(2 * ctr + 1));
    const double u1 = (double)((a >> 11) + 1) * 0x1.0p-53;  // (0, 1]
    const double u2 = (double)(b >> 11) * 0x1.0p-53;        // [0, 1)
    const double r = sqrt(-log(u1));  // sqrt(-2 ln u1) times the 1/sqrt(2) of E|w|^2 = 1
    double sn, cs;
    sincos(2.0 * M_PI * u2, &sn, &cs);
    return make_double2(r * cs, r * sn);
}

struct RsJob {
    int64_t tau, sig;    // first row / column point (global tree-order index)
    int64_t m3, n3;      // rows, columns
    int64_t a_off;       // A (m3 x n3, col-major) in the A buffer
    int64_t o_off;       // Omega (n3 x L) in the round buffer
    int64_t y_off;       // Y (m3 x L) in the round buffer
    int64_t q_off;       // Q (m3 x l) in the round buffer
    uint64_t key;
    int32_t l, prob;     // samples; problem (Green parameters)
};

// A of each job, and ||A||_F^2 (one y-row of the grid per job).
__global__ void __launch_bounds__(RS_THREADS) rs_assemble_kernel(const RsJob* jobs,
                                                                 const GreenParams* gps,
                                                                 const double* pts,
                                                                 const double* nrm, double2* A,
                                                                 double* anorm2) {
    __shared__ double red[RS_THREADS / 32];
    const RsJob J = jobs[blockIdx.y];
    const GreenParams gp = gps[J.prob];
    const int64_t m = J.m3 / 3, n = J.n3 / 3, np = m * n;
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)RS_THREADS + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * RS_THREADS) {
        const int64_t i = p % m, j = p / m;
        double2 G[9];
        entry_block(gp, pts, nrm, J.tau + i, J.sig + j, G);
        double2* col = A + J.a_off + 3 * i + 3 * j * J.m3;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const double2 g = G[3 * a + b];
                col[a + b * J.m3] = g;
                acc += g.x * g.x + g.y * g.y;
            }
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < RS_THREADS / 32; ++w) s += red[w];
        atomicAdd(anorm2 + blockIdx.y, s);
    }
}

// Omega (n3 x (l + p)) of each job.
__global__ void __launch_bounds__(RS_THREADS) rs_omega_kernel(const RsJob* jobs, double2* R) {
    const RsJob J = jobs[blockIdx.y];
    const int64_t L = J.l + RS_P, ne = J.n3 * L;
    for (int64_t e = blockIdx.x * (int64_t)RS_THREADS + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * RS_THREADS) {
        const int64_t j = e % J.n3, c = e / J.n3;
        R[J.o_off + e] = rs_gauss(J.key, (uint64_t)j * RS_CSTRIDE + (uint64_t)c);
    }
}

__device__ __forceinline__ void cmad(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

// C = op(A) B per job, FP64 complex; op(A) = A (M x K, ld lda) or A^H (A is
// K x M, ld lda).  One CTA per 32 x 32 tile of C; grid.y = job.
struct GemmJob {
    const double2* A;
    const double2* B;
    double2* C;
    int64_t M, N, K, lda, ldb, ldc;
    int32_t conj_a, pad_;
};
__global__ void __launch_bounds__(RS_THREADS) rs_gemm_kernel(const GemmJob* jobs) {
    __shared__ double2 sa[GK][GT + 1];
    __shared__ double2 sb[GK][GT + 1];
    const GemmJob J = jobs[blockIdx.y];
    const int64_t tm = (J.M + GT - 1) / GT, tn = (J.N + GT - 1) / GT;
    if ((int64_t)blockIdx.x >= tm * tn) return;
    const int64_t r0 = (blockIdx.x % tm) * GT, c0 = (blockIdx.x / tm) * GT;
    const int tid = threadIdx.x;
    const int tr = tid % 16, tc = tid / 16;  // 2 x 2 outputs: rows tr, tr + 16; columns tc, tc + 16
    double2 acc[2][2] = {};
    for (int64_t k0 = 0; k0 < J.K; k0 += GK) {
        for (int e = tid; e < GK * GT; e += RS_THREADS) {
            // op(A)(r0 + rr, k0 + kk), the stored matrix's contiguous index fastest
            const int kk = J.conj_a ? e % GK : e / GT, rr = J.conj_a ? e / GK : e % GT;
            const int64_t r = r0 + rr, k = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (r < J.M && k < J.K) {
                if (J.conj_a) {
                    v = J.A[k + r * J.lda];
                    v.y = -v.y;
                } else {
                    v = J.A[r + k * J.lda];
                }
            }
            sa[kk][rr] = v;
            const int kb = e % GK, cc = e / GK;  // B(k0 + kb, c0 + cc)
            const int64_t kq = k0 + kb, c = c0 + cc;
            sb[kb][cc] = (kq < J.K && c < J.N) ? J.B[kq + c * J.ldb] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            const double2 a0 = sa[kk][tr], a1 = sa[kk][tr + 16];
            const double2 b0 = sb[kk][tc], b1 = sb[kk][tc + 16];
            cmad(acc[0][0], a0, b0);
            cmad(acc[0][1], a0, b1);
            cmad(acc[1][0], a1, b0);
            cmad(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int64_t r = r0 + tr + 16 * i, c = c0 + tc + 16 * j;
            if (r < J.M && c < J.N) J.C[r + c * J.ldc] = acc[i][j];
        }
}

__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < RS_THREADS / 32; ++w) s += red[w];
    return s;
}

// y_c -= tau v (v^H y_c) for the columns c in [c_begin, c_end) of Y (ld m3),
// v = Y[k:, vcol] (or the explicit vector vp), rows k .. m3 - 1: a warp per column.
__device__ void apply_reflector(const double2* v, double tau, int64_t k, int64_t m3, double2* Y,
                                int64_t ldy, int64_t c_begin, int64_t c_end) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c = c_begin + warp; c < c_end; c += RS_THREADS / 32) {
        double2* y = Y + c * ldy;
        double2 w = make_double2(0.0, 0.0);
        for (int64_t r = k + lane; r < m3; r += 32) {  // w = v^H y
            const double2 a = v[r], b = y[r];
            w.x += a.x * b.x + a.y * b.y;
            w.y += a.x * b.y - a.y * b.x;
        }
        w.x = warp_sum(w.x);
        w.y = warp_sum(w.y);
        w.x *= tau;
        w.y *= tau;
        for (int64_t r = k + lane; r < m3; r += 32) {  // y -= v w
            const double2 a = v[r];
            y[r].x -= a.x * w.x - a.y * w.y;
            y[r].y -= a.x * w.y + a.y * w.x;
        }
    }
}

// One CTA per job: Householder QR of Y's first l columns (reflectors applied
// to all l + p columns, v_k kept in Y[k:, k]), the probe estimate, Q formed.
__global__ void __launch_bounds__(RS_THREADS) rs_qr_kernel(const RsJob* jobs, double2* R,
                                                           const double* anorm2, double eps,
                                                           int32_t* certified) {
    extern __shared__ double rs_tau[];  // l taus
    __shared__ double red[RS_THREADS / 32];
    const RsJob J = jobs[blockIdx.x];
    const int64_t m3 = J.m3, L = J.l + RS_P;
    double2* Y = R + J.y_off;
    for (int64_t k = 0; k < J.l; ++k) {
        double2* x = Y + k * m3;
        double s = 0.0;
        for (int64_t r = k + threadIdx.x; r < m3; r += RS_THREADS) s += x[r].x * x[r].x + x[r].y * x[r].y;
        const double nx2 = block_sum(s, red);
        double tau = 0.0;
        if (nx2 > 0.0) {
            const double2 x0 = x[k];
            const double a0 = sqrt(x0.x * x0.x + x0.y * x0.y), nx = sqrt(nx2);
            // alpha = -e^{i arg x0} ||x||; v = x - alpha e_1
            const double2 ph = a0 > 0.0 ? make_double2(x0.x / a0, x0.y / a0) : make_double2(1.0, 0.0);
            const double2 v0 = make_double2(x0.x + ph.x * nx, x0.y + ph.y * nx);
            const double vn2 = nx2 - a0 * a0 + (v0.x * v0.x + v0.y * v0.y);
            tau = 2.0 / vn2;
            __syncthreads();
            if (threadIdx.x == 0) x[k] = v0;
        }
        if (threadIdx.x == 0) rs_tau[k] = tau;
        __syncthreads();
        if (tau != 0.0) apply_reflector(x, tau, k, m3, Y, m3, k + 1, L);
        __syncthreads();
    }
    // probes: rows l .. m3 - 1 of the reflected probe columns are (I - QQ^H) A w
    double s = 0.0;
    for (int64_t c = J.l; c < L; ++c)
        for (int64_t r = J.l + threadIdx.x; r < m3; r += RS_THREADS)
            s += Y[r + c * m3].x * Y[r + c * m3].x + Y[r + c * m3].y * Y[r + c * m3].y;
    const double est = block_sum(s, red) / RS_P;
    if (threadIdx.x == 0) certified[blockIdx.x] = est <= (eps / 4) * (eps / 4) * anorm2[blockIdx.x];
    // Q = H_0 ... H_{l-1} [I; 0], accumulated backwards
    double2* Q = R + J.q_off;
    for (int64_t e = threadIdx.x; e < m3 * J.l; e += RS_THREADS) {
        const int64_t r = e % m3, c = e / m3;
        Q[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int64_t k = J.l - 1; k >= 0; --k) {
        if (rs_tau[k] != 0.0) apply_reflector(Y + k * m3, rs_tau[k], k, m3, Q, m3, k, J.l);
        __syncthreads();
    }
}

template <typename T>
T* dev_array(std::vector<DevBuf>& owner, const std::vector<T>& h, cudaStream_t st) {
    T* d = (T*)hm_dmalloc(owner, std::max<size_t>(h.size(), 1) * sizeof(T), st, false);
    HM_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return d;
}

void launch_gemm(std::vector<GemmJob>& g, std::vector<DevBuf>& tmp, cudaStream_t st) {
    if (g.empty()) return;
    int64_t tiles = 1;
    for (const GemmJob& j : g) tiles = std::max(tiles, ((j.M + GT - 1) / GT) * ((j.N + GT - 1) / GT));
    GemmJob* d = dev_array(tmp, g, st);
    rs_gemm_kernel<<<dim3((unsigned)tiles, (unsigned)g.size()), RS_THREADS, 0, st>>>(d);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
}

}  // namespace

uint64_t rsvd_key(int64_t tau_begin, int64_t sigma_begin) {
    return splitmix64(((uint64_t)tau_begin << 32) ^ (uint64_t)sigma_begin);
}

double2* rsvd_factors(std::vector<RsvdBlock>& blocks, const GreenParams* d_gps, const double* d_pts,
                      const double* d_nrm, double eps, std::vector<DevBuf>& owner, cudaStream_t st) {
    const size_t nb = blocks.size();
    if (!nb) return nullptr;
    double2* d_work = nullptr;
    std::vector<DevBuf> keep;  // A and the rounds' buffers live until the factors are out
    try {
        std::vector<RsJob> J(nb);
        int64_t aoff = 0;
        for (size_t b = 0; b < nb; ++b) {
            const RsvdBlock& B = blocks[b];
            RsJob& j = J[b];
            j.tau = B.tau_global;
            j.sig = B.sig_global;
            j.m3 = 3 * B.m;
            j.n3 = 3 * B.n;
            j.a_off = aoff;
            aoff += j.m3 * j.n3;
            j.key = B.key;
            j.prob = B.prob;
            j.l = (int32_t)std::min<int64_t>({(int64_t)RS_L0, j.m3, j.n3, (int64_t)RS_LMAX});
            j.o_off = j.y_off = j.q_off = 0;
        }
        double2* A = (double2*)hm_dmalloc(keep, (size_t)aoff * 16, st, false);
        double* anorm2 = (double*)hm_dmalloc(keep, nb * sizeof(double), st, true);
        {
            RsJob* d = dev_array(keep, J, st);
            rs_assemble_kernel<<<dim3(64, (unsigned)nb), RS_THREADS, 0, st>>>(d, d_gps, d_pts, d_nrm, A,
                                                                               anorm2);
            HM_CUDA(cudaGetLastError());
            HM_LAUNCHED();
        }
        std::vector<double2*> qfinal(nb, nullptr);
        std::vector<size_t> active(nb);
        for (size_t b = 0; b < nb; ++b) active[b] = b;
        while (!active.empty()) {
            // round buffers: Omega, Y, Q of the active jobs
            std::vector<RsJob> R;
            int64_t off = 0;
            int lmax = 1;
            for (size_t b : active) {
                RsJob j = J[b];
                const int64_t L = j.l + RS_P;
                j.o_off = off;
                off += j.n3 * L;
                j.y_off = off;
                off += j.m3 * L;
                j.q_off = off;
                off += j.m3 * j.l;
                lmax = std::max(lmax, (int)j.l);
                R.push_back(j);
            }
            double2* buf = (double2*)hm_dmalloc(keep, (size_t)off * 16, st, false);
            RsJob* d = dev_array(keep, R, st);
            rs_omega_kernel<<<dim3(32, (unsigned)R.size()), RS_THREADS, 0, st>>>(d, buf);
            HM_CUDA(cudaGetLastError());
            HM_LAUNCHED();
            std::vector<GemmJob> g;
            for (const RsJob& j : R) {  // Y = A Omega
                GemmJob q;
                q.A = A + j.a_off;
                q.B = buf + j.o_off;
                q.C = buf + j.y_off;
                q.M = j.m3;
                q.N = j.l + RS_P;
                q.K = j.n3;
                q.lda = j.m3;
                q.ldb = j.n3;
                q.ldc = j.m3;
                q.conj_a = 0;
                q.pad_ = 0;
                g.push_back(q);
            }
            launch_gemm(g, keep, st);
            std::vector<double> an(R.size());
            std::vector<double> anh(nb);
            HM_CUDA(cudaMemcpyAsync(anh.data(), anorm2, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaStreamSynchronize(st));
            for (size_t q = 0; q < R.size(); ++q) an[q] = anh[active[q]];
            double* d_an = dev_array(keep, an, st);
            int32_t* d_cert = (int32_t*)hm_dmalloc(keep, R.size() * 4, st, true);
            const size_t smem = (size_t)lmax * sizeof(double);
            rs_qr_kernel<<<(unsigned)R.size(), RS_THREADS, smem, st>>>(d, buf, d_an, eps, d_cert);
            HM_CUDA(cudaGetLastError());
            HM_LAUNCHED();
            std::vector<int32_t> cert(R.size());
            HM_CUDA(cudaMemcpyAsync(cert.data(), d_cert, R.size() * 4, cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaStreamSynchronize(st));
            std::vector<size_t> next;
            for (size_t q = 0; q < R.size(); ++q) {
                const size_t b = active[q];
                const int64_t cap = std::min<int64_t>({J[b].m3, J[b].n3, (int64_t)RS_LMAX});
                if (cert[q] || J[b].l >= cap) {
                    qfinal[b] = buf + R[q].q_off;
                    blocks[b].certified = cert[q] != 0;
                    blocks[b].l = J[b].l;
                } else {
                    J[b].l = (int32_t)std::min<int64_t>(2 * (int64_t)J[b].l, cap);
                    next.push_back(b);
                }
            }
            active.swap(next);
        }
        // U = Q and V = A^H Q into the factor workspace at the blocks' offsets
        int64_t woff = 0;
        for (size_t b = 0; b < nb; ++b) {
            blocks[b].u_off = woff;
            woff += J[b].m3 * blocks[b].l;
            blocks[b].v_off = woff;
            woff += J[b].n3 * blocks[b].l;
        }
        d_work = (double2*)hm_dmalloc(owner, (size_t)std::max<int64_t>(woff, 1) * 16, st, false);
        std::vector<GemmJob> g;
        for (size_t b = 0; b < nb; ++b) {
            const RsvdBlock& B = blocks[b];
            HM_CUDA(cudaMemcpyAsync(d_work + B.u_off, qfinal[b], (size_t)J[b].m3 * B.l * 16,
                                    cudaMemcpyDeviceToDevice, st));
            GemmJob q;
            q.A = A + J[b].a_off;
            q.B = qfinal[b];
            q.C = d_work + B.v_off;
            q.M = J[b].n3;
            q.N = B.l;
            q.K = J[b].m3;
            q.lda = J[b].m3;
            q.ldb = J[b].m3;
            q.ldc = J[b].n3;
            q.conj_a = 1;
            q.pad_ = 0;
            g.push_back(q);
        }
        launch_gemm(g, keep, st);
        HM_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        cudaStreamSynchronize(st);
        for (DevBuf& d : keep) cudaFree(d.p);
        throw;
    }
    for (DevBuf& d : keep) cudaFree(d.p);
    return d_work;
}

// gmres.cu — restarted GMRES(m) on the H-matrix (Sec. 3.1: the H-matvec is
// the only operation the iterative solver needs).  FP64 vectors on the
// device.  The Arnoldi products use the fast product (FP32 sums); the true
// residual at each restart uses the accurate product (FP64 sums over the same
// stored entries), so each restart cycle is one step of iterative refinement
// and the solve reaches tolerances below the FP32 summation noise.
// Arnoldi by classical Gram-Schmidt with one re-orthogonalisation
// (two passes of h = V^H w, w -= V h); complex Givens rotations and the least
// squares update run in a one-thread kernel, so the only host traffic per
// iteration is the 8-byte residual estimate.  x_0 = 0; convergence is
// decided on the true residual ||b - A_H x|| / ||b|| at each restart.
#include <cmath>
#include <vector>

#include "hm_internal.h"

namespace {

constexpr int GT = 256;

__global__ void to_c64_kernel(const double2* x, float2* y, int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) y[q] = make_float2((float)x[q].x, (float)x[q].y);
}

// out[i] += sum_q conj(V[q, i]) w[q], i < ncol, over a slice of rows.
__global__ void __launch_bounds__(GT) multidot_kernel(const double2* V, int64_t ld, int ncol,
                                                      const double2* w, int64_t n,
                                                      int64_t rows_per_cta, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r0 = blockIdx.x * rows_per_cta;
    const int64_t r1 = min(n, r0 + rows_per_cta);
    for (int i = wid; i < ncol; i += GT / 32) {
        double re = 0.0, im = 0.0;
        const double2* Vi = V + (int64_t)i * ld;
        for (int64_t q = r0 + lane; q < r1; q += 32) {
            const double2 v = Vi[q], x = w[q];
            re += v.x * x.x + v.y * x.y;
            im += v.x * x.y - v.y * x.x;
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) {
            atomicAdd(out + 2 * i, re);
            atomicAdd(out + 2 * i + 1, im);
        }
    }
}

// w[q] -= sum_i V[q, i] h[i]   (sign = -1), or x[q] += sum_i V[q, i] y[i] (sign = +1)
__global__ void __launch_bounds__(GT) gemv_update_kernel(const double2* V, int64_t ld, int ncol,
                                                         const double* h, double sign,
                                                         double2* w, int64_t n) {
    __shared__ double2 hs[512];
    for (int i = threadIdx.x; i < ncol; i += GT) hs[i] = make_double2(h[2 * i], h[2 * i + 1]);
    __syncthreads();
    const int64_t q = blockIdx.x * (int64_t)GT + threadIdx.x;
    if (q >= n) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < ncol; ++i) cfma(acc, V[q + (int64_t)i * ld], hs[i]);
    w[q] = make_double2(w[q].x + sign * acc.x, w[q].y + sign * acc.y);
}

__global__ void __launch_bounds__(GT) norm2_kernel(const double2* w, int64_t n, double* out) {
    double s = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)GT + threadIdx.x; q < n; q += (int64_t)gridDim.x * GT)
        s += cabs2(w[q]);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// dst = a * src + b * dst2  (general axpby into dst)
__global__ void axpby_kernel(double2* dst, const double2* src, double a, const double2* src2,
                             double b, int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) {
        const double2 u = src[q], v = src2[q];
        dst[q] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
    }
}

// v = w / sqrt(nrm2[0])
__global__ void scale_kernel(double2* v, const double2* w, const double* nrm2, int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double s = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
    if (q < n) v[q] = cscale(w[q], s);
}

struct GState {
    double* H;    // (m+1) x m complex, col-major
    double* cs;   // m complex
    double* sn;   // m complex
    double* g;    // m+1 complex
    double* y;    // m complex
    double* h1;   // m+1 complex (first pass)
    double* h2;   // m+1 complex (second pass)
    double* nrm2; // scalar
    double* est;  // |g_{j+1}| (host-read)
};

// H[:, j] = h1 + h2 (0..j), H[j+1, j] = sqrt(nrm2); previous rotations; new rotation.
__global__ void givens_kernel(GState S, int m, int j) {
    auto Hc = [&](int i) { return reinterpret_cast<double2*>(S.H) + i + (int64_t)j * (m + 1); };
    double2* cs = reinterpret_cast<double2*>(S.cs);
    double2* sn = reinterpret_cast<double2*>(S.sn);
    double2* g = reinterpret_cast<double2*>(S.g);
    const double2* h1 = reinterpret_cast<const double2*>(S.h1);
    const double2* h2 = reinterpret_cast<const double2*>(S.h2);
    for (int i = 0; i <= j; ++i) *Hc(i) = cadd(h1[i], h2[i]);
    *Hc(j + 1) = make_double2(sqrt(S.nrm2[0]), 0.0);
    for (int i = 0; i < j; ++i) {
        const double2 a = *Hc(i), b = *Hc(i + 1);
        *Hc(i) = cadd(cmul(cs[i], a), cmul(sn[i], b));
        *Hc(i + 1) = cadd(cscale(cmul(cconj(sn[i]), a), -1.0), cmul(cs[i], b));
    }
    const double2 a = *Hc(j), b = *Hc(j + 1);
    const double aa = sqrt(cabs2(a)), nu = sqrt(cabs2(a) + cabs2(b));
    if (aa == 0.0) {
        cs[j] = make_double2(0.0, 0.0);
        sn[j] = make_double2(1.0, 0.0);
    } else {
        cs[j] = make_double2(aa / nu, 0.0);
        sn[j] = cscale(cmul(make_double2(a.x / aa, a.y / aa), cconj(b)), 1.0 / nu);
    }
    *Hc(j) = cadd(cmul(cs[j], a), cmul(sn[j], b));
    *Hc(j + 1) = make_double2(0.0, 0.0);
    const double2 g0 = g[j];
    g[j] = cmul(cs[j], g0);
    g[j + 1] = cscale(cmul(cconj(sn[j]), g0), -1.0);
    S.est[0] = sqrt(cabs2(g[j + 1]));
}

__global__ void backsolve_kernel(GState S, int m, int jend) {
    const double2* H = reinterpret_cast<const double2*>(S.H);
    const double2* g = reinterpret_cast<const double2*>(S.g);
    double2* y = reinterpret_cast<double2*>(S.y);
    for (int i = jend - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int q = i + 1; q < jend; ++q) acc = csub(acc, cmul(H[i + (int64_t)q * (m + 1)], y[q]));
        y[i] = cdiv(acc, H[i + (int64_t)i * (m + 1)]);
    }
}

__global__ void init_g_kernel(double* g, const double* nrm2, int m) {
    for (int i = 0; i < 2 * (m + 1); ++i) g[i] = 0.0;
    g[0] = sqrt(nrm2[0]);
}

}  // namespace

// y = A_H x for FP64 vectors (tree-order work vectors of the handle).
static void apply_fp64(hm_matrix* h, const double2* x, double2* y, cudaStream_t st) {
    matvec_graph(h->mv, h->d_perm, x, h->d_xp, h->d_yp, y, h->nc, st);
}

GmresResult gmres_solve(hm_matrix* h, const double2* b, double2* x, int m, double tol, int maxit,
                        cudaStream_t st) {
    const int64_t n = 3 * h->nc;
    const unsigned nb = (unsigned)hm_cdiv(n, GT);
    std::vector<DevBuf> tmp;
    auto dm = [&](size_t bytes) { return hm_dmalloc(tmp, bytes, st, true); };
    double2* Vb = (double2*)dm((size_t)n * (m + 1) * sizeof(double2));
    double2* w = (double2*)dm((size_t)n * sizeof(double2));
    GState S;
    S.H = (double*)dm((size_t)2 * (m + 1) * m * sizeof(double));
    S.cs = (double*)dm((size_t)2 * m * sizeof(double));
    S.sn = (double*)dm((size_t)2 * m * sizeof(double));
    S.g = (double*)dm((size_t)2 * (m + 1) * sizeof(double));
    S.y = (double*)dm((size_t)2 * m * sizeof(double));
    S.h1 = (double*)dm((size_t)2 * (m + 1) * sizeof(double));
    S.h2 = (double*)dm((size_t)2 * (m + 1) * sizeof(double));
    S.nrm2 = (double*)dm(sizeof(double));
    S.est = (double*)dm(sizeof(double));
    double2* xp64 = (double2*)dm((size_t)n * sizeof(double2));
    double2* yp64 = (double2*)dm((size_t)n * sizeof(double2));
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        for (DevBuf& d : tmp) cudaFree(d.p);
        tmp.clear();
    };
    GmresResult R{0, 1.0, 0};
    try {
        const int64_t rows_per = 4096;
        const unsigned ndot = (unsigned)hm_cdiv(n, rows_per);
        auto nrm2_of = [&](const double2* v) {
            HM_CUDA(cudaMemsetAsync(S.nrm2, 0, sizeof(double), st));
            norm2_kernel<<<std::min<unsigned>(nb, 1024), GT, 0, st>>>(v, n, S.nrm2);
            HM_LAUNCHED();
            HM_CUDA(cudaGetLastError());
            double v2 = 0.0;
            HM_CUDA(cudaMemcpyAsync(&v2, S.nrm2, sizeof(double), cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaStreamSynchronize(st));
            return v2;
        };
        HM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), st));
        const double bn = std::sqrt(nrm2_of(b));
        if (bn == 0.0) {
            R.relres = 0.0;
            R.converged = 1;
            cleanup();
            return R;
        }
        int iters = 0;
        for (;;) {
            // r = b - A x with the accurate product (iterative refinement of the
            // fast FP32 inner iterations), into V_0
            matvec_accurate(h->mv, h->d_perm, x, xp64, yp64, w, h->nc, st);
            axpby_kernel<<<nb, GT, 0, st>>>(w, b, 1.0, w, -1.0, n);
            HM_LAUNCHED();
            HM_CUDA(cudaGetLastError());
            const double beta2 = nrm2_of(w);
            R.relres = std::sqrt(beta2) / bn;
            if (R.relres <= tol) {
                R.converged = 1;
                break;
            }
            if (iters >= maxit) break;
            scale_kernel<<<nb, GT, 0, st>>>(Vb, w, S.nrm2, n);
            HM_LAUNCHED();
            init_g_kernel<<<1, 1, 0, st>>>(S.g, S.nrm2, m);
            HM_LAUNCHED();
            HM_CUDA(cudaGetLastError());
            int jend = 0;
            for (int j = 0; j < m; ++j) {
                apply_fp64(h, Vb + (int64_t)j * n, w, st);
                iters++;
                for (int pass = 0; pass < 2; ++pass) {
                    double* hh = pass == 0 ? S.h1 : S.h2;
                    HM_CUDA(cudaMemsetAsync(hh, 0, 2 * (j + 1) * sizeof(double), st));
                    multidot_kernel<<<ndot, GT, 0, st>>>(Vb, n, j + 1, w, n, rows_per, hh);
                    HM_LAUNCHED();
                    gemv_update_kernel<<<nb, GT, 0, st>>>(Vb, n, j + 1, hh, -1.0, w, n);
                    HM_LAUNCHED();
                    HM_CUDA(cudaGetLastError());
                }
                HM_CUDA(cudaMemsetAsync(S.nrm2, 0, sizeof(double), st));
                norm2_kernel<<<std::min<unsigned>(nb, 1024), GT, 0, st>>>(w, n, S.nrm2);
                HM_LAUNCHED();
                scale_kernel<<<nb, GT, 0, st>>>(Vb + (int64_t)(j + 1) * n, w, S.nrm2, n);
                HM_LAUNCHED();
                givens_kernel<<<1, 1, 0, st>>>(S, m, j);
                HM_LAUNCHED();
                HM_CUDA(cudaGetLastError());
                double est = 0.0, hn2 = 0.0;
                HM_CUDA(cudaMemcpyAsync(&est, S.est, sizeof(double), cudaMemcpyDeviceToHost, st));
                HM_CUDA(cudaMemcpyAsync(&hn2, S.nrm2, sizeof(double), cudaMemcpyDeviceToHost, st));
                HM_CUDA(cudaStreamSynchronize(st));
                jend = j + 1;
                if (!(est == est)) hm_throw(HM_ERR_NUMERIC, "GMRES produced a non-finite residual");
                if (est / bn <= tol || iters >= maxit || hn2 == 0.0) break;
            }
            backsolve_kernel<<<1, 1, 0, st>>>(S, m, jend);
            HM_LAUNCHED();
            gemv_update_kernel<<<nb, GT, 0, st>>>(Vb, n, jend, S.y, 1.0, x, n);
            HM_LAUNCHED();
            HM_CUDA(cudaGetLastError());
        }
        R.iters = iters;
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
    return R;
}

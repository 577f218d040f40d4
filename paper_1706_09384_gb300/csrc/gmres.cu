// gmres.cu — restarted GMRES(m) on the H-matrix (Sec. 3.1: the H-matvec is
// the only operation the iterative solver needs).  FP64 vectors on the
// device.  The Arnoldi products use the fast product (FP32 sums); the true
// residual at each restart uses the accurate product (double-float sums of
// about 44 significant bits over the same stored entries), so each restart
// cycle is one step of iterative refinement and the solve reaches tolerances
// below the FP32 summation noise.
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
__device__ void givens_step(const GState& S, int m, int j) {
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

__global__ void givens_kernel(GState S, int m, int j) { givens_step(S, m, j); }

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


// ---- several right-hand sides in lockstep (blockIdx.y = right-hand side s) ----
// Basis vector j of right-hand side s: V + (j * nrhs + s) * n; w_s = W + s * n;
// per-right-hand-side scalars at stride `hs` (complex) in h, one flag per s in act.

__global__ void __launch_bounds__(GT) multidot_b_kernel(const double2* V, int nrhs, int ncol,
                                                        const double2* W, int64_t n,
                                                        int64_t rows_per_cta, double* out,
                                                        int hs, const int* act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r0 = blockIdx.x * rows_per_cta;
    const int64_t r1 = min(n, r0 + rows_per_cta);
    const double2* w = W + (int64_t)s * n;
    for (int i = wid; i < ncol; i += GT / 32) {
        double re = 0.0, im = 0.0;
        const double2* Vi = V + ((int64_t)i * nrhs + s) * n;
        for (int64_t q = r0 + lane; q < r1; q += 32) {
            const double2 v = Vi[q], x = w[q];
            re += v.x * x.x + v.y * x.y;
            im += v.x * x.y - v.y * x.x;
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) {
            atomicAdd(out + 2 * ((int64_t)s * hs + i), re);
            atomicAdd(out + 2 * ((int64_t)s * hs + i) + 1, im);
        }
    }
}

// w_s -= sum_i V_{i,s} h_{s,i} (sign -1, ncol columns) or x_s += sum_i V_{i,s} y_{s,i}
// (sign +1, ncol_of[s] columns when ncol_of is given)
__global__ void __launch_bounds__(GT) gemv_update_b_kernel(const double2* V, int nrhs, int ncol,
                                                           const int* ncol_of, const double* h,
                                                           int hs, double sign, double2* W,
                                                           int64_t n, const int* act) {
    const int s = blockIdx.y;
    if (act && !act[s]) return;
    const int nc = ncol_of ? ncol_of[s] : ncol;
    __shared__ double2 hsh[512];
    for (int i = threadIdx.x; i < nc; i += GT)
        hsh[i] = make_double2(h[2 * ((int64_t)s * hs + i)], h[2 * ((int64_t)s * hs + i) + 1]);
    __syncthreads();
    const int64_t q = blockIdx.x * (int64_t)GT + threadIdx.x;
    if (q >= n) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < nc; ++i) cfma(acc, V[((int64_t)i * nrhs + s) * n + q], hsh[i]);
    double2* w = W + (int64_t)s * n;
    w[q] = make_double2(w[q].x + sign * acc.x, w[q].y + sign * acc.y);
}

__global__ void __launch_bounds__(GT) norm2_b_kernel(const double2* W, int64_t n, double* out,
                                                     const int* act) {
    const int s = blockIdx.y;
    if (act && !act[s]) return;
    const double2* w = W + (int64_t)s * n;
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)GT + threadIdx.x; q < n; q += (int64_t)gridDim.x * GT)
        acc += cabs2(w[q]);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) atomicAdd(out + s, acc);
}

// V_{j,s} = w_s / sqrt(nrm2[s])
__global__ void scale_b_kernel(double2* V, int nrhs, int j, const double2* W, const double* nrm2,
                               int64_t n, const int* act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double f = nrm2[s] > 0.0 ? 1.0 / sqrt(nrm2[s]) : 0.0;
    if (q < n) V[((int64_t)j * nrhs + s) * n + q] = cscale(W[(int64_t)s * n + q], f);
}

// w_s = b_s - w_s for the unconverged right-hand sides
__global__ void residual_b_kernel(double2* W, const double2* B, int64_t n, const int* act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) {
        const double2 b = B[(int64_t)s * n + q], w = W[(int64_t)s * n + q];
        W[(int64_t)s * n + q] = make_double2(b.x - w.x, b.y - w.y);
    }
}

struct GStateB {
    double* H;    // per s: (m+1) x m complex, col-major
    double* cs;   // per s: m complex
    double* sn;
    double* g;    // per s: m+1 complex
    double* y;    // per s: m complex
    double* h1;   // per s: m+1 complex
    double* h2;
    double* nrm2; // per s
    double* est;  // per s
};

__global__ void givens_b_kernel(GStateB S, int m, int j, const int* act) {
    const int s = blockIdx.x;
    if (!act[s]) return;
    GState T;
    T.H = S.H + (int64_t)s * 2 * (m + 1) * m;
    T.cs = S.cs + (int64_t)s * 2 * m;
    T.sn = S.sn + (int64_t)s * 2 * m;
    T.g = S.g + (int64_t)s * 2 * (m + 1);
    T.y = S.y + (int64_t)s * 2 * m;
    T.h1 = S.h1 + (int64_t)s * 2 * (m + 1);
    T.h2 = S.h2 + (int64_t)s * 2 * (m + 1);
    T.nrm2 = S.nrm2 + s;
    T.est = S.est + s;
    givens_step(T, m, j);
}

__global__ void backsolve_b_kernel(GStateB S, int m, const int* jend) {
    const int s = blockIdx.x;
    const int je = jend[s];
    const double2* H = reinterpret_cast<const double2*>(S.H) + (int64_t)s * (m + 1) * m;
    const double2* g = reinterpret_cast<const double2*>(S.g) + (int64_t)s * (m + 1);
    double2* y = reinterpret_cast<double2*>(S.y) + (int64_t)s * m;
    for (int i = je - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int q = i + 1; q < je; ++q) acc = csub(acc, cmul(H[i + (int64_t)q * (m + 1)], y[q]));
        y[i] = cdiv(acc, H[i + (int64_t)i * (m + 1)]);
    }
}

__global__ void init_g_b_kernel(double* g, const double* nrm2, int m, const int* act) {
    const int s = blockIdx.x;
    if (!act[s]) return;
    double* gs = g + (int64_t)s * 2 * (m + 1);
    for (int i = 0; i < 2 * (m + 1); ++i) gs[i] = 0.0;
    gs[0] = sqrt(nrm2[s]);
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
        for (bool first = true;; first = false) {
            // r = b - A x with the accurate product (iterative refinement of the
            // fast FP32 inner iterations), into V_0; r = b for x_0 = 0
            if (first) {
                HM_CUDA(cudaMemcpyAsync(w, b, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            } else {
                matvec_accurate(h->mv, h->d_perm, x, xp64, yp64, w, h->nc, st);
                axpby_kernel<<<nb, GT, 0, st>>>(w, b, 1.0, w, -1.0, n);
                HM_LAUNCHED();
                HM_CUDA(cudaGetLastError());
            }
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

// Several right-hand sides in lockstep: one restarted GMRES per right-hand
// side, all sharing each fast product (a block product on the tensor cores
// with BF16 storage, else one product per column).  A right-hand side whose
// residual estimate reaches tol is frozen for the rest of its cycle; the true
// residuals (accurate products) at each restart decide convergence.
void gmres_solve_multi(hm_matrix* h, int nrhs, const double2* B, double2* X, int m, double tol,
                       int maxit, std::vector<GmresResult>& out, cudaStream_t st) {
    const int64_t n = 3 * h->nc;
    const unsigned nb = (unsigned)hm_cdiv(n, GT);
    std::vector<DevBuf> tmp;
    auto dm = [&](size_t bytes) { return hm_dmalloc(tmp, bytes, st, true); };
    double2* Vb = (double2*)dm((size_t)n * (m + 1) * nrhs * sizeof(double2));
    double2* W = (double2*)dm((size_t)n * nrhs * sizeof(double2));
    GStateB S;
    S.H = (double*)dm((size_t)2 * (m + 1) * m * nrhs * sizeof(double));
    S.cs = (double*)dm((size_t)2 * m * nrhs * sizeof(double));
    S.sn = (double*)dm((size_t)2 * m * nrhs * sizeof(double));
    S.g = (double*)dm((size_t)2 * (m + 1) * nrhs * sizeof(double));
    S.y = (double*)dm((size_t)2 * m * nrhs * sizeof(double));
    S.h1 = (double*)dm((size_t)2 * (m + 1) * nrhs * sizeof(double));
    S.h2 = (double*)dm((size_t)2 * (m + 1) * nrhs * sizeof(double));
    S.nrm2 = (double*)dm((size_t)nrhs * sizeof(double));
    S.est = (double*)dm((size_t)nrhs * sizeof(double));
    int* d_act = (int*)dm((size_t)nrhs * sizeof(int));
    int* d_jend = (int*)dm((size_t)nrhs * sizeof(int));
    double2* xp64 = (double2*)dm((size_t)n * sizeof(double2));
    double2* yp64 = (double2*)dm((size_t)n * sizeof(double2));
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        for (DevBuf& d : tmp) cudaFree(d.p);
        tmp.clear();
    };
    out.assign(nrhs, GmresResult{0, 1.0, 0});
    try {
        const int64_t rows_per = 4096;
        const unsigned ndot = (unsigned)hm_cdiv(n, rows_per);
        const dim3 gv(nb, nrhs), gd(ndot, nrhs), gn(std::min<unsigned>(nb, 256), nrhs);
        std::vector<int> act(nrhs, 1), jend(nrhs, 0);
        std::vector<double> hv(nrhs), hest(nrhs), bn(nrhs);
        auto upload_act = [&]() {
            HM_CUDA(cudaMemcpyAsync(d_act, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
        };
        auto norms = [&](const double2* V) {  // nrm2[s] = ||V_s||^2 for active s, to the host
            HM_CUDA(cudaMemsetAsync(S.nrm2, 0, nrhs * sizeof(double), st));
            norm2_b_kernel<<<gn, GT, 0, st>>>(V, n, S.nrm2, d_act);
            HM_LAUNCHED();
            HM_CUDA(cudaGetLastError());
            HM_CUDA(cudaMemcpyAsync(hv.data(), S.nrm2, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaStreamSynchronize(st));
        };
        HM_CUDA(cudaMemsetAsync(X, 0, (size_t)n * nrhs * sizeof(double2), st));
        upload_act();
        norms(B);
        for (int s = 0; s < nrhs; ++s) {
            bn[s] = std::sqrt(hv[s]);
            if (bn[s] == 0.0) {
                out[s].relres = 0.0;
                out[s].converged = 1;
            }
        }
        int iters = 0;
        for (bool first = true;; first = false) {
            // true residuals of the unconverged right-hand sides (accurate
            // products; W = A X = 0 for X_0 = 0)
            for (int s = 0; s < nrhs; ++s) act[s] = !out[s].converged;
            upload_act();
            if (first) {
                HM_CUDA(cudaMemsetAsync(W, 0, (size_t)n * nrhs * sizeof(double2), st));
            } else {
                for (int s = 0; s < nrhs; ++s)
                    if (act[s])
                        matvec_accurate(h->mv, h->d_perm, X + (int64_t)s * n, xp64, yp64,
                                        W + (int64_t)s * n, h->nc, st);
            }
            residual_b_kernel<<<gv, GT, 0, st>>>(W, B, n, d_act);
            HM_LAUNCHED();
            HM_CUDA(cudaGetLastError());
            norms(W);
            bool any = false;
            for (int s = 0; s < nrhs; ++s) {
                if (!act[s]) continue;
                out[s].relres = std::sqrt(hv[s]) / bn[s];
                if (out[s].relres <= tol) {
                    out[s].converged = 1;
                    act[s] = 0;
                } else {
                    any = true;
                }
            }
            if (!any || iters >= maxit) break;
            upload_act();
            scale_b_kernel<<<gv, GT, 0, st>>>(Vb, nrhs, 0, W, S.nrm2, n, d_act);
            HM_LAUNCHED();
            init_g_b_kernel<<<nrhs, 1, 0, st>>>(S.g, S.nrm2, m, d_act);
            HM_LAUNCHED();
            HM_CUDA(cudaGetLastError());
            std::fill(jend.begin(), jend.end(), 0);
            for (int j = 0; j < m; ++j) {
                const double2* Vj = Vb + (int64_t)j * nrhs * n;
                if (h->opts.storage == HM_STORE_BF16 && nrhs > 1) {
                    matvec_multi(h->mv, h->d_perm, Vj, W, h->nc, nrhs, st);
                } else {
                    for (int s = 0; s < nrhs; ++s)
                        if (act[s])
                            matvec_graph(h->mv, h->d_perm, Vj + (int64_t)s * n, h->d_xp, h->d_yp,
                                         W + (int64_t)s * n, h->nc, st);
                }
                iters++;
                for (int pass = 0; pass < 2; ++pass) {
                    double* hh = pass == 0 ? S.h1 : S.h2;
                    HM_CUDA(cudaMemsetAsync(hh, 0, (size_t)2 * (m + 1) * nrhs * sizeof(double), st));
                    multidot_b_kernel<<<gd, GT, 0, st>>>(Vb, nrhs, j + 1, W, n, rows_per, hh, m + 1,
                                                         d_act);
                    HM_LAUNCHED();
                    gemv_update_b_kernel<<<gv, GT, 0, st>>>(Vb, nrhs, j + 1, nullptr, hh, m + 1,
                                                            -1.0, W, n, d_act);
                    HM_LAUNCHED();
                    HM_CUDA(cudaGetLastError());
                }
                HM_CUDA(cudaMemsetAsync(S.nrm2, 0, nrhs * sizeof(double), st));
                norm2_b_kernel<<<gn, GT, 0, st>>>(W, n, S.nrm2, d_act);
                HM_LAUNCHED();
                scale_b_kernel<<<gv, GT, 0, st>>>(Vb, nrhs, j + 1, W, S.nrm2, n, d_act);
                HM_LAUNCHED();
                givens_b_kernel<<<nrhs, 1, 0, st>>>(S, m, j, d_act);
                HM_LAUNCHED();
                HM_CUDA(cudaGetLastError());
                HM_CUDA(cudaMemcpyAsync(hest.data(), S.est, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
                HM_CUDA(cudaMemcpyAsync(hv.data(), S.nrm2, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
                HM_CUDA(cudaStreamSynchronize(st));
                bool left = false, changed = false;
                for (int s = 0; s < nrhs; ++s) {
                    if (!act[s]) continue;
                    jend[s] = j + 1;
                    out[s].iters = iters;
                    if (!(hest[s] == hest[s]))
                        hm_throw(HM_ERR_NUMERIC, "GMRES produced a non-finite residual");
                    if (hest[s] / bn[s] <= tol || hv[s] == 0.0) {
                        act[s] = 0;
                        changed = true;
                    } else {
                        left = true;
                    }
                }
                if (!left || iters >= maxit) break;
                if (changed) upload_act();
            }
            HM_CUDA(cudaMemcpyAsync(d_jend, jend.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
            backsolve_b_kernel<<<nrhs, 1, 0, st>>>(S, m, d_jend);
            HM_LAUNCHED();
            gemv_update_b_kernel<<<gv, GT, 0, st>>>(Vb, nrhs, 0, d_jend, S.y, m, 1.0, X, n, nullptr);
            HM_LAUNCHED();
            HM_CUDA(cudaGetLastError());
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

// gmres.cu — restarted GMRES(m) on the H-matrix (Sec. 3.1: the H-matvec is
// the only operation the iterative solver needs).  FP64 vectors on the
// device.  The Arnoldi products use the fast product (FP32 or BF16 x FP32
// sums); the true residual at each restart uses the accurate product
// (double-float sums of about 44 significant bits over the FP32-stored
// entries), so each restart cycle is one step of iterative refinement and the
// solve reaches tolerances below the FP32 summation noise.
//
// One code path serves one right-hand side, nrhs of them in lockstep, and the
// independent problems of a joined batch handle (hm_batch_join: a
// block-diagonal operator whose diagonal blocks are the problems) in
// lockstep.  A solve works on "segments": segment s (blockIdx.y) is the part
// [off_s, off_s + len_s) of each vector; right-hand sides are equal-length
// segments of one column-major block, problems are the consecutive parts of
// the concatenated vector.  A flag per segment freezes the converged ones.
// With several right-hand sides each Arnoldi step makes one product of all
// of them (the tensor-core block product with BF16 storage); with a batch it
// makes one product of the block-diagonal operator, i.e. of every problem at
// once.  An Arnoldi step is the product plus four kernels:
//   dot      h1 = V^H w                       (classical Gram-Schmidt, pass 1)
//   upd_dot  w -= V h1, h2 = V^H w            (pass 2: re-orthogonalisation)
//   norm     w -= V h2, ||w||^2, then the Givens update of the Hessenberg
//            column and of the residual estimate |g_{j+1}|
//   scale    v_{j+1} = w / ||w||
// Each kernel runs on a grid of row slices sized from the SM count; a CTA
// writes its partial sums to global memory and the last CTA to finish (a
// ticket taken with one atomic, no waiting) adds them in a fixed order, so
// results do not depend on scheduling and there are no same-address
// floating-point atomics.  The scalars of the small problem (Givens rotations,
// the least-squares right-hand side) stay on the device; the host reads 16
// bytes per right-hand side per step from pinned memory to decide
// convergence.  The basis and all scratch come from the library's
// stream-ordered pool (scratch.cu), so a solve makes no cudaMalloc.  x_0 = 0;
// convergence is decided on the true residual ||b - A_H x|| / ||b|| at each
// restart.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hm_internal.h"

namespace {

constexpr int GT = 256;
constexpr int GW = GT / 32;
constexpr int MAXM = 500;  // restart length limit of the ABI
// Relative accuracy assumed for the BF16 fast product before a restart has
// measured it (the bench workloads: 1e-5 weighted, up to ~1e-3 without
// weights); a cycle's inner iteration stops at half of it times the cycle's
// starting residual, since the true residual cannot follow the fast operator
// further (iterative refinement with an inexact inner solve).
constexpr double IR_DELTA0_BF16 = 1e-4;

// Device pointers and sizes of a solve (passed by value to every kernel).
struct GP {
    int64_t N;          // length of one whole vector (all segments)
    const int64_t* off; // [s] first entry of segment s
    const int64_t* len; // [s] entries of segment s
    int m;              // restart length
    int nrhs;           // segments
    int G;              // CTAs per segment (row slices)
    double2* V;         // basis: vector j, segment s at V + j N + off_s
    double2* part;   // partial sums [s][cta][m + 1]
    double* partn;   // partial norms [s][cta]
    unsigned* cnt;   // tickets [s]
    double2* H;      // [s] (m+1) x m column-major
    double2* cs;     // [s][m]
    double2* sn;     // [s][m]
    double2* g;      // [s][m+1]
    double2* y;      // [s][m]
    double2* h1;     // [s][m+1]
    double2* h2;     // [s][m+1]
    double* nrm2;    // [s]; est[s] = nrm2[nrhs + s]
    const int* act;  // [s] 1 = column still iterating (nullptr: all)
};

HM_D double2* basis(const GP& P, int j, int s) { return P.V + (int64_t)j * P.N + P.off[s]; }

// rows [r0, r1) of segment s handled by this CTA
HM_D void cta_rows(const GP& P, int s, int64_t& r0, int64_t& r1) {
    const int64_t n = P.len[s], rpc = (n + P.G - 1) / P.G;
    r0 = min(n, (int64_t)blockIdx.x * rpc);
    r1 = min(n, r0 + rpc);
}

// The last CTA of right-hand side s to arrive returns true (after every other
// CTA's partial sums are visible); it also re-arms the ticket.
HM_D bool last_cta(const GP& P, int s) {
    __shared__ unsigned s_ticket;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = atomicAdd(P.cnt + s, 1u);
    __syncthreads();
    if (s_ticket != (unsigned)gridDim.x - 1) return false;
    __threadfence();
    if (threadIdx.x == 0) P.cnt[s] = 0;
    return true;
}

// w -= sum_{i < ncol} V_i h_i over this CTA's rows (h from global, staged in shared memory).
HM_D void update_rows(const GP& P, int s, int ncol, const double2* h, double2* w, int64_t r0,
                      int64_t r1, double2* hs) {
    for (int i = threadIdx.x; i < ncol; i += GT) hs[i] = h[(int64_t)s * (P.m + 1) + i];
    __syncthreads();
    for (int64_t q = r0 + threadIdx.x; q < r1; q += GT) {
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < ncol; ++i) cfma(acc, basis(P, i, s)[q], hs[i]);
        w[q] = make_double2(w[q].x - acc.x, w[q].y - acc.y);
    }
    __syncthreads();  // this CTA's writes to w are visible to all its threads
}

// hout[s][i] = V_i^H w for i < ncol (optionally after w -= V hsub).
__global__ void __launch_bounds__(GT) dot_kernel(GP P, int ncol, const double2* hsub,
                                                 double2* W, double2* hout) {
    const int s = blockIdx.y;
    if (P.act && !P.act[s]) return;
    __shared__ double2 hs[MAXM + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t r0, r1;
    cta_rows(P, s, r0, r1);
    double2* w = W + P.off[s];
    if (hsub) update_rows(P, s, ncol, hsub, w, r0, r1, hs);
    double2* part = P.part + ((int64_t)s * P.G + blockIdx.x) * (P.m + 1);
    for (int i = wid; i < ncol; i += GW) {
        const double2* Vi = basis(P, i, s);
        double re = 0.0, im = 0.0;
        for (int64_t q = r0 + lane; q < r1; q += 32) {
            const double2 v = Vi[q], x = w[q];
            re = fma(v.x, x.x, fma(v.y, x.y, re));
            im = fma(v.x, x.y, fma(-v.y, x.x, im));
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) part[i] = make_double2(re, im);
    }
    if (!last_cta(P, s)) return;
    const double2* ps = P.part + (int64_t)s * P.G * (P.m + 1);
    for (int i = wid; i < ncol; i += GW) {
        double re = 0.0, im = 0.0;
        for (int c = lane; c < P.G; c += 32) {
            const double2 v = __ldcg(ps + (int64_t)c * (P.m + 1) + i);
            re += v.x;
            im += v.y;
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) hout[(int64_t)s * (P.m + 1) + i] = make_double2(re, im);
    }
}

// Givens update of column j of the Hessenberg matrix of right-hand side s:
// H[:, j] = h1 + h2, H[j+1, j] = sqrt(nrm2); previous rotations; new rotation;
// est = |g_{j+1}|.
HM_D void givens_step(const GP& P, int s, int j) {
    const int m = P.m;
    double2* Hj = P.H + (int64_t)s * (m + 1) * m + (int64_t)j * (m + 1);
    double2* cs = P.cs + (int64_t)s * m;
    double2* sn = P.sn + (int64_t)s * m;
    double2* g = P.g + (int64_t)s * (m + 1);
    const double2* h1 = P.h1 + (int64_t)s * (m + 1);
    const double2* h2 = P.h2 + (int64_t)s * (m + 1);
    for (int i = 0; i <= j; ++i) Hj[i] = cadd(h1[i], h2[i]);
    Hj[j + 1] = make_double2(sqrt(P.nrm2[s]), 0.0);
    for (int i = 0; i < j; ++i) {
        const double2 a = Hj[i], b = Hj[i + 1];
        Hj[i] = cadd(cmul(cs[i], a), cmul(sn[i], b));
        Hj[i + 1] = cadd(cscale(cmul(cconj(sn[i]), a), -1.0), cmul(cs[i], b));
    }
    const double2 a = Hj[j], b = Hj[j + 1];
    const double aa = sqrt(cabs2(a)), nu = sqrt(cabs2(a) + cabs2(b));
    if (aa == 0.0) {
        cs[j] = make_double2(0.0, 0.0);
        sn[j] = make_double2(1.0, 0.0);
    } else {
        cs[j] = make_double2(aa / nu, 0.0);
        sn[j] = cscale(cmul(make_double2(a.x / aa, a.y / aa), cconj(b)), 1.0 / nu);
    }
    Hj[j] = cadd(cmul(cs[j], a), cmul(sn[j], b));
    Hj[j + 1] = make_double2(0.0, 0.0);
    const double2 g0 = g[j];
    g[j] = cmul(cs[j], g0);
    g[j + 1] = cscale(cmul(cconj(sn[j]), g0), -1.0);
    P.nrm2[P.nrhs + s] = sqrt(cabs2(g[j + 1]));
}

// nrm2[s] = ||w_s||^2, after (B != null) w = b - w and/or (hsub != null)
// w -= V hsub over ncol columns.  mode 1: then g = (sqrt(nrm2), 0, ...) (start
// of a cycle); mode 2: then the Givens update of column j.
__global__ void __launch_bounds__(GT) norm_kernel(GP P, int mode, int j, const double2* B,
                                                  const double2* hsub, int ncol, double2* W) {
    const int s = blockIdx.y;
    if (P.act && !P.act[s]) return;
    __shared__ double2 hs[MAXM + 1];
    __shared__ double red[GW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t r0, r1;
    cta_rows(P, s, r0, r1);
    double2* w = W + P.off[s];
    if (B) {
        const double2* b = B + P.off[s];
        for (int64_t q = r0 + threadIdx.x; q < r1; q += GT)
            w[q] = make_double2(b[q].x - w[q].x, b[q].y - w[q].y);
        __syncthreads();
    }
    if (hsub) update_rows(P, s, ncol, hsub, w, r0, r1, hs);
    double acc = 0.0;
    for (int64_t q = r0 + threadIdx.x; q < r1; q += GT) acc += cabs2(w[q]);
    acc = warp_sum(acc);
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < GW; ++q) t += red[q];
        P.partn[(int64_t)s * P.G + blockIdx.x] = t;
    }
    if (!last_cta(P, s)) return;
    if (wid == 0) {
        double t = 0.0;
        for (int c = lane; c < P.G; c += 32) t += __ldcg(P.partn + (int64_t)s * P.G + c);
        t = warp_sum(t);
        if (lane == 0) {
            P.nrm2[s] = t;
            if (mode == 1) {
                double2* g = P.g + (int64_t)s * (P.m + 1);
                for (int i = 0; i <= P.m; ++i) g[i] = make_double2(0.0, 0.0);
                g[0] = make_double2(sqrt(t), 0.0);
                P.nrm2[P.nrhs + s] = sqrt(t);
            } else if (mode == 2) {
                givens_step(P, s, j);
            }
        }
    }
}

// basis vector j of every active right-hand side = w_s / ||w_s||
__global__ void scale_kernel(GP P, int j, const double2* W) {
    const int s = blockIdx.y;
    if (P.act && !P.act[s]) return;
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double f = P.nrm2[s] > 0.0 ? 1.0 / sqrt(P.nrm2[s]) : 0.0;
    if (q < P.len[s]) basis(P, j, s)[q] = cscale(W[P.off[s] + q], f);
}

// w_s = b_s for the active right-hand sides (first cycle: r = b for x_0 = 0)
__global__ void copy_kernel(GP P, const double2* B, double2* W) {
    const int s = blockIdx.y;
    if (P.act && !P.act[s]) return;
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < P.len[s]) W[P.off[s] + q] = B[P.off[s] + q];
}

// y_s = R^{-1} g over the first jend[s] columns (one thread per right-hand side)
__global__ void backsolve_kernel(GP P, const int* jend) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.nrhs) return;
    const int je = jend[s], m = P.m;
    const double2* H = P.H + (int64_t)s * (m + 1) * m;
    const double2* g = P.g + (int64_t)s * (m + 1);
    double2* y = P.y + (int64_t)s * m;
    for (int i = je - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int q = i + 1; q < je; ++q) acc = csub(acc, cmul(H[i + (int64_t)q * (m + 1)], y[q]));
        y[i] = cdiv(acc, H[i + (int64_t)i * (m + 1)]);
    }
}

// x_s += sum_{i < jend[s]} V_i y_s[i]
__global__ void __launch_bounds__(GT) update_x_kernel(GP P, const int* jend, double2* X) {
    const int s = blockIdx.y;
    const int je = jend[s];
    if (je == 0) return;
    __shared__ double2 ys[MAXM];
    for (int i = threadIdx.x; i < je; i += GT) ys[i] = P.y[(int64_t)s * P.m + i];
    __syncthreads();
    const int64_t q = blockIdx.x * (int64_t)GT + threadIdx.x;
    if (q >= P.len[s]) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < je; ++i) cfma(acc, basis(P, i, s)[q], ys[i]);
    double2* x = X + P.off[s];
    x[q] = cadd(x[q], acc);
}

}  // namespace

// Workspace of one solve: scratch from the library's stream-ordered pool
// (freed memory stays in the pool, so repeated solves allocate nothing new).
struct GmresWork {
    GP P{};
    double2* W = nullptr;
    int* d_act = nullptr;
    int* d_jend = nullptr;
    double2* xp64 = nullptr;
    double2* yp64 = nullptr;
    double* host = nullptr;  // pinned: nrm2[nrhs], est[nrhs]
    int64_t lmax = 0;        // longest segment
    std::vector<void*> bufs;
    cudaStream_t st = nullptr;
    ~GmresWork() {
        for (void* p : bufs) hm_scratch_free(p, st);
        if (host) hm_pinned_give(host);
    }
};

static void gmres_work(GmresWork& g, hm_matrix* h, int m, const std::vector<int64_t>& off,
                       const std::vector<int64_t>& len, cudaStream_t st) {
    const int nrhs = (int)off.size();
    int64_t N = 0, lmax = 0;
    for (int s = 0; s < nrhs; ++s) {
        N = std::max(N, off[s] + len[s]);
        lmax = std::max(lmax, len[s]);
    }
    int nsm = 0;
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    g.st = st;
    g.lmax = lmax;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(hm_cdiv(lmax, GT), 4 * (int64_t)nsm));
    auto dm = [&](size_t bytes) {
        void* p = hm_scratch_alloc(bytes, st);
        g.bufs.push_back(p);
        return p;
    };
    GP& P = g.P;
    P.N = N;
    P.m = m;
    P.nrhs = nrhs;
    P.G = G;
    int64_t* d_seg = (int64_t*)dm((size_t)2 * nrhs * sizeof(int64_t));
    std::vector<int64_t> seg(off);
    seg.insert(seg.end(), len.begin(), len.end());
    HM_CUDA(cudaMemcpyAsync(d_seg, seg.data(), seg.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    P.off = d_seg;
    P.len = d_seg + nrhs;
    P.V = (double2*)dm((size_t)N * (m + 1) * sizeof(double2));
    P.part = (double2*)dm((size_t)nrhs * G * (m + 1) * sizeof(double2));
    P.partn = (double*)dm((size_t)nrhs * G * sizeof(double));
    P.cnt = (unsigned*)dm((size_t)nrhs * sizeof(unsigned));
    HM_CUDA(cudaMemsetAsync(P.cnt, 0, (size_t)nrhs * sizeof(unsigned), st));
    P.H = (double2*)dm((size_t)nrhs * (m + 1) * m * sizeof(double2));
    P.cs = (double2*)dm((size_t)nrhs * m * sizeof(double2));
    P.sn = (double2*)dm((size_t)nrhs * m * sizeof(double2));
    P.g = (double2*)dm((size_t)nrhs * (m + 1) * sizeof(double2));
    P.y = (double2*)dm((size_t)nrhs * m * sizeof(double2));
    P.h1 = (double2*)dm((size_t)nrhs * (m + 1) * sizeof(double2));
    P.h2 = (double2*)dm((size_t)nrhs * (m + 1) * sizeof(double2));
    P.nrm2 = (double*)dm((size_t)2 * nrhs * sizeof(double));
    g.d_act = (int*)dm((size_t)nrhs * sizeof(int));
    P.act = g.d_act;
    g.d_jend = (int*)dm((size_t)nrhs * sizeof(int));
    g.W = (double2*)dm((size_t)N * sizeof(double2));
    g.xp64 = (double2*)dm((size_t)3 * h->nc * sizeof(double2));
    g.yp64 = (double2*)dm((size_t)3 * h->nc * sizeof(double2));
    g.host = (double*)hm_pinned_take((size_t)2 * nrhs * sizeof(double));
}

// Restarted GMRES per segment of B, run in lockstep.  Columns mode: segment s
// is right-hand side s (equal lengths 3 n_c, column-major B); each Arnoldi
// step makes one fast product of all active columns (a block product on the
// tensor cores with BF16 storage and several columns, else one product per
// column).  Segments mode (a joined batch handle): segment s is problem s of
// the block-diagonal operator and each step makes one product of the whole
// vector.  A segment is frozen for the rest of its cycle when its residual
// estimate reaches max(tol ||b||, delta ||r_c|| / 2): r_c is the true residual
// at the cycle's start and delta the relative accuracy of the fast product
// (0 with FP32 storage; with BF16 the prior above, raised to the reduction a
// cycle actually achieved when that is worse), since below delta ||r_c|| the
// fast operator's error, not the Krylov space, limits the true residual.  The
// true residuals (accurate products) at each restart decide convergence.
static void gmres_core(hm_matrix* h, bool columns, const std::vector<int64_t>& off,
                       const std::vector<int64_t>& len, const double2* B, double2* X, int m,
                       double tol, int maxit, std::vector<GmresResult>& out, cudaStream_t st) {
    const int nrhs = (int)off.size();
    const int64_t n = 3 * h->nc;
    GmresWork work;
    gmres_work(work, h, m, off, len, st);
    GmresWork* gw = &work;
    // one product covers every segment, frozen ones included: their part of the
    // basis must hold numbers (the pool returns uninitialised memory)
    if (!columns)
        HM_CUDA(cudaMemsetAsync(work.P.V, 0, (size_t)work.P.N * (m + 1) * sizeof(double2), st));
    GP P = gw->P;
    double2* W = gw->W;
    h->gm_fast = h->gm_accurate = h->gm_cycles = 0;
    const unsigned nb = (unsigned)hm_cdiv(gw->lmax, GT);
    const dim3 gv(nb, nrhs), gd((unsigned)P.G, nrhs);
    out.assign(nrhs, GmresResult{0, 1.0, 0});
    std::vector<int> act(nrhs, 1), jend(nrhs, 0);
    std::vector<double> bn(nrhs, 0.0);
    // inner stopping thresholds (absolute) and the fast product's accuracy per segment
    std::vector<double> thr(nrhs, 0.0), prev_rel(nrhs, 1.0);
    std::vector<double> delta(nrhs, h->opts.storage == HM_STORE_BF16 ? IR_DELTA0_BF16 : 0.0);
    double* hv = gw->host;           // nrm2 per segment
    double* hest = gw->host + nrhs;  // residual estimate per segment
    // segments mode: the products skip the work items of frozen segments (the
    // full item lists come back when the solve ends, also on an error)
    std::vector<int64_t> bounds(off);
    bounds.push_back(P.N);
    struct Restore {
        hm_matrix* h;
        const std::vector<int64_t>* b;
        cudaStream_t st;
        bool on;
        ~Restore() {
            if (!on) return;
            try {
                matvec_select_segments(h->mv, *b, std::vector<int>(b->size() - 1, 1), st);
            } catch (...) {
            }
        }
    } restore{h, &bounds, st, !columns};
    std::vector<int> sel_act;
    auto upload_act = [&]() {  // pageable source: safe to modify after the call returns
        HM_CUDA(cudaMemcpyAsync(gw->d_act, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
        if (!columns && act != sel_act) {
            matvec_select_segments(h->mv, bounds, act, st);
            sel_act = act;
        }
    };
    auto readback = [&]() {
        HM_CUDA(cudaMemcpyAsync(gw->host, P.nrm2, 2 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
    };
    auto launched = [&]() {
        HM_LAUNCHED();
        HM_CUDA(cudaGetLastError());
    };
    HM_CUDA(cudaMemsetAsync(X, 0, (size_t)P.N * sizeof(double2), st));
    upload_act();
    // ||b_s||: the norm kernel on a copy of B
    copy_kernel<<<gv, GT, 0, st>>>(P, B, W);
    launched();
    norm_kernel<<<gd, GT, 0, st>>>(P, 0, 0, nullptr, nullptr, 0, W);
    launched();
    readback();
    for (int s = 0; s < nrhs; ++s) {
        bn[s] = std::sqrt(hv[s]);
        if (bn[s] == 0.0) {
            out[s].relres = 0.0;
            out[s].converged = 1;
        }
    }
    int iters = 0;
    for (bool first = true;; first = false) {
        // true residuals of the unconverged segments (accurate products; r = b for x_0 = 0)
        for (int s = 0; s < nrhs; ++s) act[s] = !out[s].converged;
        upload_act();
        if (first) {
            copy_kernel<<<gv, GT, 0, st>>>(P, B, W);
            launched();
            norm_kernel<<<gd, GT, 0, st>>>(P, 1, 0, nullptr, nullptr, 0, W);
        } else {
            if (columns) {
                for (int s = 0; s < nrhs; ++s)
                    if (act[s]) {
                        matvec_accurate(h->mv, h->d_perm, X + off[s], gw->xp64, gw->yp64, W + off[s],
                                        h->nc, st);
                        h->gm_accurate++;
                    }
            } else {
                matvec_accurate(h->mv, h->d_perm, X, gw->xp64, gw->yp64, W, h->nc, st);
                h->gm_accurate++;
            }
            norm_kernel<<<gd, GT, 0, st>>>(P, 1, 0, B, nullptr, 0, W);
        }
        launched();
        readback();
        bool any = false;
        for (int s = 0; s < nrhs; ++s) {
            if (!act[s]) continue;
            out[s].relres = std::sqrt(hv[s]) / bn[s];
            if (!(out[s].relres == out[s].relres))
                hm_throw(HM_ERR_NUMERIC, "GMRES produced a non-finite residual");
            if (out[s].relres <= tol) {
                out[s].converged = 1;
                act[s] = 0;
            } else {
                any = true;
                if (!first && delta[s] > 0.0) delta[s] = std::max(delta[s], out[s].relres / prev_rel[s]);
                prev_rel[s] = out[s].relres;
                thr[s] = std::max(tol, 0.5 * delta[s] * out[s].relres) * bn[s];
            }
        }
        if (!any || iters >= maxit) break;
        upload_act();
        scale_kernel<<<gv, GT, 0, st>>>(P, 0, W);
        launched();
        h->gm_cycles++;
        std::fill(jend.begin(), jend.end(), 0);
        for (int j = 0; j < m; ++j) {
            double2* Vj = P.V + (int64_t)j * P.N;
            if (!columns) {
                matvec_graph(h->mv, h->d_perm, Vj, h->d_xp, h->d_yp, W, h->nc, st);
                h->gm_fast++;
            } else if (h->opts.storage == HM_STORE_BF16 && nrhs > 1) {
                matvec_multi(h->mv, h->d_perm, Vj, W, h->nc, nrhs, st);
                h->gm_fast += nrhs;
            } else {
                for (int s = 0; s < nrhs; ++s)
                    if (act[s]) {
                        matvec_graph(h->mv, h->d_perm, Vj + off[s], h->d_xp, h->d_yp, W + off[s],
                                     h->nc, st);
                        h->gm_fast++;
                    }
            }
            iters++;
            dot_kernel<<<gd, GT, 0, st>>>(P, j + 1, nullptr, W, P.h1);
            launched();
            dot_kernel<<<gd, GT, 0, st>>>(P, j + 1, P.h1, W, P.h2);
            launched();
            norm_kernel<<<gd, GT, 0, st>>>(P, 2, j, nullptr, P.h2, j + 1, W);
            launched();
            scale_kernel<<<gv, GT, 0, st>>>(P, j + 1, W);
            launched();
            readback();
            bool left = false, changed = false;
            for (int s = 0; s < nrhs; ++s) {
                if (!act[s]) continue;
                jend[s] = j + 1;
                out[s].iters = iters;
                if (!(hest[s] == hest[s]))
                    hm_throw(HM_ERR_NUMERIC, "GMRES produced a non-finite residual");
                if (hest[s] <= thr[s] || hv[s] == 0.0) {
                    act[s] = 0;
                    changed = true;
                } else {
                    left = true;
                }
            }
            if (!left || iters >= maxit) break;
            if (changed) upload_act();
        }
        HM_CUDA(cudaMemcpyAsync(gw->d_jend, jend.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
        backsolve_kernel<<<(unsigned)hm_cdiv(nrhs, 32), 32, 0, st>>>(P, gw->d_jend);
        launched();
        update_x_kernel<<<gv, GT, 0, st>>>(P, gw->d_jend, X);
        launched();
    }
    (void)n;
}

void gmres_solve_multi(hm_matrix* h, int nrhs, const double2* B, double2* X, int m, double tol,
                       int maxit, std::vector<GmresResult>& out, cudaStream_t st) {
    const int64_t n = 3 * h->nc;
    std::vector<int64_t> off(nrhs), len(nrhs, n);
    for (int s = 0; s < nrhs; ++s) off[s] = s * n;
    gmres_core(h, true, off, len, B, X, m, tol, maxit, out, st);
}

void gmres_solve_segments(hm_matrix* h, const std::vector<int64_t>& seg_points, const double2* B,
                          double2* X, int m, double tol, int maxit, std::vector<GmresResult>& out,
                          cudaStream_t st) {
    std::vector<int64_t> off, len;
    int64_t o = 0;
    for (int64_t p : seg_points) {
        off.push_back(3 * o);
        len.push_back(3 * p);
        o += p;
    }
    if (o != h->nc) hm_throw(HM_ERR_ARG, "segments do not cover the handle's points");
    gmres_core(h, false, off, len, B, X, m, tol, maxit, out, st);
}

GmresResult gmres_solve(hm_matrix* h, const double2* b, double2* x, int m, double tol, int maxit,
                        cudaStream_t st) {
    std::vector<GmresResult> R;
    gmres_solve_multi(h, 1, b, x, m, tol, maxit, R, st);
    return R[0];
}

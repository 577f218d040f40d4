// recompress.cu — recompression of the ACA factors (Sec. 3.2).
//
// The paper writes B = U V^H = Q_U R_U R_V^H Q_V^H, takes the SVD
// R_U R_V^H = P S L^H and keeps U' = Q_U P S^{1/2}, V' = Q_V L S^{1/2}
// truncated with eps_ACA.  Here the triangular factors come from the Gram
// matrices (U^H U = R_U^H R_U, a Cholesky factorisation of the equilibrated
// Gram matrix, semi-definite: a non-positive pivot zeroes its row), and the
// orthonormal factors are never formed: from R_U R_V^H L = P S and
// (R_U R_V^H)^H P = L S,
//     Q_U P_r S_r^{1/2} = U (R_V^H L_r S_r^{-1/2}) =: U T_U,
//     Q_V L_r S_r^{1/2} = V (R_U^H P_r S_r^{-1/2}) =: V T_V,
// which holds whether or not R_U, R_V are invertible.  The Gram matrices, their
// Cholesky factors and the core W are FP64; the SVD of the k x k core is a
// one-sided Jacobi (Hestenes) iteration in double-float arithmetic on the FP32
// pipes (approximate angles, exactly unitary rotations) with round-robin pair ordering.  Truncation:
// smallest r' with
// (sum_{i >= r'} s_i^2)^{1/2} <= eps (sum s_i^2)^{1/2} (Frobenius, matching the
// ACA stopping test).  The tall products U T_U, V T_V are applied by a second
// kernel, in double-float arithmetic on the FP32 pipes (~44 significant bits
// before the rounding to the FP32 storage), that writes straight into the
// matvec's chunk layout.
#include <algorithm>

#include "hm_internal.h"

namespace {

constexpr int RT = 256;

// complex128 -> double-float pair (re_hi, im_hi, re_lo, im_lo): the T factors
// are handed to the factor application in this form (same 16 bytes)
__device__ __forceinline__ float4 to_df(double2 v) {
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
}
constexpr int RW = RT / 32;
constexpr int TILE_ROWS = 16;

struct CoreJob {
    int64_t u_off, v_off;   // workspace offsets of U (m3 x k), V (n3 x k)
    int64_t m3, n3;
    int64_t s_off;          // scratch offset: 6 k^2 complex
    int64_t g_off;          // Gram matrices from the ACA (G_U then G_V, ld g_ld), or -1
    int32_t g_ld;
    int32_t k;
    int32_t recompress;
    int32_t pad_;
};

// G = A^H A for a col-major (rows x k) A, into G (k x k col-major).
__device__ void gram(const double2* A, int64_t rows, int k, double2* G, double2* tile) {
    const int tid = threadIdx.x;
    const int64_t nent = (int64_t)k * k;
    constexpr int EPT = 8;  // entries per thread per pass
    for (int64_t e0 = 0; e0 < nent; e0 += (int64_t)RT * EPT) {
        double2 acc[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) acc[q] = make_double2(0.0, 0.0);
        for (int64_t r0 = 0; r0 < rows; r0 += TILE_ROWS) {
            __syncthreads();
            const int tr = (int)(rows - r0 < TILE_ROWS ? rows - r0 : TILE_ROWS);
            for (int t = tid; t < TILE_ROWS * k; t += RT) {
                const int c = t / TILE_ROWS, r = t - c * TILE_ROWS;
                tile[c * TILE_ROWS + r] = r < tr ? A[r0 + r + (int64_t)c * rows] : make_double2(0.0, 0.0);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int64_t e = e0 + (int64_t)q * RT + tid;
                if (e < nent) {
                    const int p = (int)(e % k), c = (int)(e / k);
                    if (p <= c) {
                        const double2* tp = tile + p * TILE_ROWS;
                        const double2* tc = tile + c * TILE_ROWS;
#pragma unroll
                        for (int r = 0; r < TILE_ROWS; ++r) cfma_conja(acc[q], tp[r], tc[r]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int64_t e = e0 + (int64_t)q * RT + tid;
            if (e < nent) {
                const int p = (int)(e % k), c = (int)(e / k);
                if (p <= c) {
                    G[p + (int64_t)c * k] = acc[q];
                    if (p != c) G[c + (int64_t)p * k] = cconj(acc[q]);
                }
            }
        }
    }
    __syncthreads();
}

// In place: G (Hermitian PSD, k x k col-major) -> R upper with G = R^H R, after
// equilibration G' = D^-1 G D^-1 (D = sqrt diag G); R = R' D.  Serial over
// columns, parallel over the trailing entries.
__device__ void chol_equil(double2* G, int k, double* dsc) {
    const int tid = threadIdx.x;
    for (int j = tid; j < k; j += RT) {
        const double d = G[j + (int64_t)j * k].x;
        dsc[j] = d > 0.0 ? sqrt(d) : 0.0;
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)k * k; e += RT) {
        const int p = (int)(e % k), c = (int)(e / k);
        const double s = (dsc[p] > 0.0 && dsc[c] > 0.0) ? 1.0 / (dsc[p] * dsc[c]) : 0.0;
        G[e] = cscale(G[e], s);
    }
    __syncthreads();
    // right-looking Cholesky on the upper triangle: G = R^H R
    __shared__ double s_piv;
    for (int j = 0; j < k; ++j) {
        if (tid == 0) {
            const double d = G[j + (int64_t)j * k].x;
            s_piv = d > 1e-13 ? sqrt(d) : 0.0;
        }
        __syncthreads();
        const double piv = s_piv;
        // row j of R: R_jc = G_jc / piv for c > j
        for (int c = j + 1 + tid; c < k; c += RT)
            G[j + (int64_t)c * k] = piv > 0.0 ? cscale(G[j + (int64_t)c * k], 1.0 / piv) : make_double2(0.0, 0.0);
        if (tid == 0) G[j + (int64_t)j * k] = make_double2(piv, 0.0);
        __syncthreads();
        // trailing update: G_ab -= conj(R_ja) R_jb for j < a <= b
        const int64_t nt = (int64_t)(k - j - 1) * (k - j - 1);
        for (int64_t e = tid; e < nt; e += RT) {
            const int a = j + 1 + (int)(e % (k - j - 1)), b = j + 1 + (int)(e / (k - j - 1));
            if (a <= b) {
                const double2 ra = G[j + (int64_t)a * k], rb = G[j + (int64_t)b * k];
                double2 g = G[a + (int64_t)b * k];
                cfms_conja(g, ra, rb);  // g -= conj(ra) rb, fused
                G[a + (int64_t)b * k] = g;
            }
        }
        __syncthreads();
    }
    // zero the strict lower triangle, scale columns: R = R' D
    for (int64_t e = tid; e < (int64_t)k * k; e += RT) {
        const int p = (int)(e % k), c = (int)(e / k);
        G[e] = p > c ? make_double2(0.0, 0.0) : cscale(G[e], dsc[c]);
    }
    __syncthreads();
}

// ---- double-float arithmetic for the core's Jacobi (pairs of FP32 numbers,
// about 2^-46 relative; Dekker's product with an FMA, Knuth's two-sum; every
// operation explicitly rounded so nothing is fused) ----
struct dfl {
    float h, l;
};
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ dfl df_norm(float h, float l) {  // |l| small against |h|
    const float s = __fadd_rn(h, l);
    return {s, __fsub_rn(l, __fsub_rn(s, h))};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const dfl s = df_two_sum(a.h, b.h);
    return df_norm(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_norm(p, e);
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }
// s += a b (accumulating; a, b double-float)
__device__ __forceinline__ void df_acc(float& h, float& l, dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const dfl t = df_two_sum(h, p);
    h = t.h;
    l = __fadd_rn(l, __fadd_rn(t.l, e));
}
// 1 / sqrt(a) for a > 0 in double-float: the FP32 estimate refined by one
// Newton step x + x (1 - a x^2) / 2 evaluated in double-float (relative error
// about 2^-43, from the estimate's 2^-22 squared)
__device__ __forceinline__ dfl df_rsqrt(dfl a) {
    const float x = rsqrtf(a.h);
    const float x2 = __fmul_rn(x, x);
    const dfl xx = df_norm(x2, __fmaf_rn(x, x, -x2));  // x^2 exactly
    const dfl d = df_add({1.f, 0.f}, df_neg(df_mul(a, xx)));
    const dfl corr = df_mul(d, {0.5f * x, 0.f});
    return df_add({x, 0.f}, corr);
}
__device__ __forceinline__ dfl df_scale(dfl a, float p2) { return {a.h * p2, a.l * p2}; }  // p2 a power of 2
__device__ __forceinline__ double2 from_df(float4 v) {
    return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

// One-sided (Hestenes) Jacobi on the columns of the k x k core W (entries as
// double-float pairs (re_h, im_h, re_l, im_l)), round-robin pair ordering.
// Each pair is handled by a group of G lanes (G grows with k): the lanes form
// the pair's Gram entries as double-float dot products, the group leader turns
// them into the rotation (tangent in FP32, the unitary factors in double-float)
// and broadcasts it, and the lanes apply it in double-float.  Only the final columns P_j s_j are needed (T_U, T_V below), so
// the rotations are not accumulated.  The truncation formulas map the
// rounding of the small columns through W^H, which amplifies it by up to
// (s_1 / s_r)^2 ~ eps^-2: the arithmetic must keep u << eps^2 (FP32 does not;
// double-float does for eps >= 1e-6).  A pair is rotated while
// |<w_a, w_b>| > 1e-12 ||w_a|| ||w_b||; at most 40 sweeps.
__device__ void jacobi_columns_df(float4* W, int k) {
    __shared__ int s_conv;
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = k <= 128 ? 8 : (k <= 256 ? 16 : 32);
    const int gl = lane % G;                // lane within the group
    const int gid = tid / G;                // group index in the CTA
    const int ngroups = RT / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - gl));
    const int np = (k + 1) & ~1;  // players (a dummy when k is odd)
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (tid == 0) s_conv = 1;
        __syncthreads();
        for (int round = 0; round < np - 1; ++round) {
            for (int pi = gid; pi < np / 2; pi += ngroups) {
                int a, b;
                if (pi == 0) {
                    a = np - 1;
                    b = round;
                } else {
                    a = (round + pi) % (np - 1);
                    b = (round - pi + np - 1) % (np - 1);
                }
                if (a >= k || b >= k) continue;  // uniform within the group
                float s[8] = {};  // alpha, beta, Re g, Im g as (h, l) pairs; g = <w_a, w_b>
                for (int r = gl; r < k; r += G) {
                    const float4 wa = W[r + (int64_t)a * k], wb = W[r + (int64_t)b * k];
                    const dfl ar = {wa.x, wa.z}, ai = {wa.y, wa.w}, br = {wb.x, wb.z}, bi = {wb.y, wb.w};
                    df_acc(s[0], s[1], ar, ar);
                    df_acc(s[0], s[1], ai, ai);
                    df_acc(s[2], s[3], br, br);
                    df_acc(s[2], s[3], bi, bi);
                    df_acc(s[4], s[5], ar, br);          // Re conj(wa) wb
                    df_acc(s[4], s[5], ai, bi);
                    df_acc(s[6], s[7], ar, bi);          // Im conj(wa) wb
                    df_acc(s[6], s[7], df_neg(ai), br);
                }
                for (int o = G / 2; o > 0; o >>= 1)  // group sums, double-float
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const dfl u = {__shfl_xor_sync(gmask, s[2 * q], o),
                                       __shfl_xor_sync(gmask, s[2 * q + 1], o)};
                        const dfl t = df_add({s[2 * q], s[2 * q + 1]}, u);
                        s[2 * q] = t.h;
                        s[2 * q + 1] = t.l;
                    }
                // Rotation parameters on the group leader, without FP64: the
                // tangent t may be approximate (FP32, on values scaled by a power
                // of two), but the applied rotation must be unitary to double-float
                // precision, so c = 1 / sqrt(1 + t^2), s = c t and the phase
                // e^{-i phi} = conj(g) / |g| are formed in double-float arithmetic.
                dfl dc = {1.f, 0.f}, ds = {0.f, 0.f}, dpr = {1.f, 0.f}, dpi = {0.f, 0.f};
                int rot = 0;
                if (gl == 0) {
                    const dfl al = {s[0], s[1]}, be = {s[2], s[3]}, gr = {s[4], s[5]}, gi = {s[6], s[7]};
                    const float gmax = fmaxf(fabsf(gr.h), fabsf(gi.h));
                    const float nmax = fmaxf(al.h, be.h);
                    if (gmax > 0.f && nmax > 0.f) {
                        // |g|^2 > 1e-24 al be on scaled values (norms to <= 1, g to [1, 2))
                        const float sn = scalbnf(1.f, -ilogbf(nmax));
                        const float sg = scalbnf(1.f, -ilogbf(gmax));
                        const dfl grs = df_scale(gr, sg), gis = df_scale(gi, sg);
                        const float ag = sqrtf(grs.h * grs.h + gis.h * gis.h) * (sn / sg);  // |g| sn
                        const float als = al.h * sn, bes = be.h * sn;
                        if (ag > 0.f && ag * ag > 1e-24f * als * bes) {
                            rot = 1;
                            const float zeta = (bes - als) / (2.f * ag);
                            const float az = fabsf(zeta);
                            const float t = (zeta >= 0.f ? 1.f : -1.f) /
                                            (az > 1e18f ? 2.f * az : az + sqrtf(1.f + az * az));
                            const float t2 = __fmul_rn(t, t);
                            dc = df_rsqrt(df_add({1.f, 0.f}, df_norm(t2, __fmaf_rn(t, t, -t2))));
                            ds = df_mul(dc, {t, 0.f});
                            const dfl g2 = df_add(df_mul(grs, grs), df_mul(gis, gis));
                            const dfl inv = df_rsqrt(g2);
                            dpr = df_mul(grs, inv);
                            dpi = df_neg(df_mul(gis, inv));
                        }
                    }
                }
                const int src = lane - gl;
                rot = __shfl_sync(gmask, rot, src);
                if (!rot) continue;
                dc = {__shfl_sync(gmask, dc.h, src), __shfl_sync(gmask, dc.l, src)};
                ds = {__shfl_sync(gmask, ds.h, src), __shfl_sync(gmask, ds.l, src)};
                dpr = {__shfl_sync(gmask, dpr.h, src), __shfl_sync(gmask, dpr.l, src)};
                dpi = {__shfl_sync(gmask, dpi.h, src), __shfl_sync(gmask, dpi.l, src)};
                if (gl == 0) s_conv = 0;
                // [w_a, w_b] <- [w_a, w_b] [[c, s], [-s e^{-i phi}, c e^{-i phi}]]
                for (int r = gl; r < k; r += G) {
                    const float4 wa = W[r + (int64_t)a * k], wb = W[r + (int64_t)b * k];
                    const dfl ar = {wa.x, wa.z}, ai = {wa.y, wa.w}, br = {wb.x, wb.z}, bi = {wb.y, wb.w};
                    // pw = e^{-i phi} w_b
                    const dfl pwr = df_add(df_mul(dpr, br), df_neg(df_mul(dpi, bi)));
                    const dfl pwi = df_add(df_mul(dpr, bi), df_mul(dpi, br));
                    const dfl nar = df_add(df_mul(dc, ar), df_neg(df_mul(ds, pwr)));
                    const dfl nai = df_add(df_mul(dc, ai), df_neg(df_mul(ds, pwi)));
                    const dfl nbr = df_add(df_mul(ds, ar), df_mul(dc, pwr));
                    const dfl nbi = df_add(df_mul(ds, ai), df_mul(dc, pwi));
                    W[r + (int64_t)a * k] = make_float4(nar.h, nai.h, nar.l, nai.l);
                    W[r + (int64_t)b * k] = make_float4(nbr.h, nbi.h, nbr.l, nbi.l);
                }
            }
            __syncthreads();
        }
        if (s_conv) break;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(RT) recomp_core_kernel(const CoreJob* jobs, double2* work,
                                                         const double2* gram_in, double2* scratch,
                                                         double eps, int32_t* rank_out,
                                                         int tile_cap) {
    extern __shared__ double2 tile[];       // TILE_ROWS x k
    __shared__ double dsc[1024];
    __shared__ int s_r;
    const CoreJob J = jobs[blockIdx.x];
    const int k = J.k;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (k == 0) {
        if (tid == 0) rank_out[blockIdx.x] = 0;
        return;
    }
    double2* RU = scratch + J.s_off;
    double2* RV = RU + (int64_t)k * k;
    double2* W = RV + (int64_t)k * k;
    double2* L = W + (int64_t)k * k;
    double2* TU = L + (int64_t)k * k;
    double2* TV = TU + (int64_t)k * k;
    if (!J.recompress) {
        for (int64_t e = tid; e < (int64_t)k * k; e += RT) {
            const int p = (int)(e % k), c = (int)(e / k);
            const float4 one = to_df(make_double2(p == c ? 1.0 : 0.0, 0.0));
            reinterpret_cast<float4*>(TU)[e] = one;
            reinterpret_cast<float4*>(TV)[e] = one;
        }
        if (tid == 0) rank_out[blockIdx.x] = k;
        return;
    }
    if (gram_in && J.g_off >= 0) {  // G_U, G_V accumulated by the ACA
        const double2* GU = gram_in + J.g_off;
        const double2* GV = GU + (int64_t)J.g_ld * J.g_ld;
        for (int64_t e = tid; e < (int64_t)k * k; e += RT) {
            const int p = (int)(e % k), c = (int)(e / k);
            RU[e] = GU[p + (int64_t)c * J.g_ld];
            RV[e] = GV[p + (int64_t)c * J.g_ld];
        }
        __syncthreads();
    } else {
        gram(work + J.u_off, J.m3, k, RU, tile);
        gram(work + J.v_off, J.n3, k, RV, tile);
    }
    double2* GVc = L;  // keep G_V = V^H V: T_U is formed from it after the SVD
    for (int64_t e = tid; e < (int64_t)k * k; e += RT) GVc[e] = RV[e];
    __syncthreads();
    chol_equil(RU, k, dsc);
    chol_equil(RV, k, dsc);
    // W = R_U R_V^H (the k x k core)
    for (int64_t e = tid; e < (int64_t)k * k; e += RT) {
        const int p = (int)(e % k), c = (int)(e / k);
        double2 acc = make_double2(0.0, 0.0);
        for (int t = max(p, c); t < k; ++t)  // R_U[p][t] nonzero for t >= p, R_V[c][t] for t >= c
            cfma_conjb(acc, RU[p + (int64_t)t * k], RV[c + (int64_t)t * k]);  // acc += a conj(b)
        W[e] = acc;
    }
    __syncthreads();
    // The k x k core's SVD: one-sided Jacobi in double-float arithmetic on W,
    // converted in place (16 bytes per entry either way).
    float4* Wd = reinterpret_cast<float4*>(W);
    for (int64_t e = tid; e < (int64_t)k * k; e += RT) Wd[e] = to_df(W[e]);
    __syncthreads();
    jacobi_columns_df(Wd, k);
    // singular values (column norms) and descending order
    __shared__ double s_sv[1024];
    __shared__ int s_ord[1024];
    for (int j = wid; j < k; j += RW) {
        double a = 0.0;
        for (int r = lane; r < k; r += 32) a += cabs2(from_df(Wd[r + (int64_t)j * k]));
        a = warp_sum(a);
        if (lane == 0) s_sv[j] = sqrt(a);
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = 0; j < k; ++j) s_ord[j] = j;
        for (int i = 0; i < k; ++i) {  // selection sort, ties keep index order
            int best = i;
            for (int j = i + 1; j < k; ++j)
                if (s_sv[s_ord[j]] > s_sv[s_ord[best]]) best = j;
            const int t = s_ord[i];
            s_ord[i] = s_ord[best];
            s_ord[best] = t;
        }
        double tot = 0.0;
        for (int j = 0; j < k; ++j) tot += s_sv[j] * s_sv[j];
        int r = k;
        double tail = 0.0;
        for (int i = k - 1; i >= 0; --i) {
            const double sv = s_sv[s_ord[i]];
            if (sqrt(tail + sv * sv) <= eps * sqrt(tot)) {
                tail += sv * sv;
                r = i;
            } else {
                break;
            }
        }
        s_r = r;
        rank_out[blockIdx.x] = r;
    }
    __syncthreads();
    const int r = s_r;
    // With M = R_U R_V^H = P S L^H:  M M^H P = P S^2  and  M^H P = L S, so
    //   T_V = R_U^H P_r S_r^{-1/2}                  (V' = V T_V = Q_V L_r S_r^{1/2})
    //   T_U = G_V T_V S_r^{-1} = R_V^H L_r S_r^{-1/2} (U' = U T_U = Q_U P_r S_r^{1/2}),
    // with P_j = W_j / s_j and G_V = V^H V = R_V^H R_V.
    for (int64_t e = tid; e < (int64_t)k * r; e += RT) {
        const int p = (int)(e % k), q = (int)(e / k);
        const int j = s_ord[q];
        const double s = s_sv[j];
        double2 av = make_double2(0.0, 0.0);
        for (int t = 0; t <= p; ++t)  // (R_U^H)_{p t} = conj(R_U[t][p]), nonzero for t <= p
            cfma_conja(av, RU[t + (int64_t)p * k], from_df(Wd[t + (int64_t)j * k]));
        TV[p + (int64_t)q * k] = cscale(av, 1.0 / (s * sqrt(s)));
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)k * r; e += RT) {
        const int p = (int)(e % k), q = (int)(e / k);
        const double s = s_sv[s_ord[q]];
        double2 au = make_double2(0.0, 0.0);
        for (int t = 0; t < k; ++t) cfma(au, GVc[p + (int64_t)t * k], TV[t + (int64_t)q * k]);
        TU[p + (int64_t)q * k] = cscale(au, 1.0 / s);
    }
    __syncthreads();
    // T_U, T_V as double-float pairs, in place, for the factor application
    for (int64_t e = tid; e < (int64_t)k * r; e += RT) {
        reinterpret_cast<float4*>(TU)[e] = to_df(TU[e]);
        reinterpret_cast<float4*>(TV)[e] = to_df(TV[e]);
    }
}

// One item = the rows of one leaf of one factor.
struct ApplyJob {
    int64_t src;     // workspace offset of the leaf's first row in the factor (m3 x k)
    int64_t src_ld;  // factor rows
    int64_t t_off;   // scratch offset of T (k x r, ld k)
    int64_t dst;     // arena offset of the chunk
    int32_t k, r, rows, ld;
};

// U' = U T on FP32 pipes: U (complex128) is split into a double-float pair on
// load, T arrives as double-float pairs; each complex multiply-add is four
// double-float multiply-adds (the high product split exactly by an FMA, the
// cross terms and the rounding errors gathered in the low word, exact
// two-sums), good to about 2^-44 before the final rounding to FP32.
__device__ __forceinline__ void df_mac(float& h, float& l, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float t = __fadd_rn(h, p);
    const float bp = __fsub_rn(t, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    h = t;
    l = __fadd_rn(l, __fadd_rn(err, e));
}

// With HAS_DF the factor is read from the ACA's double-float copy (the same
// split as below, made once when the column was written), so no FP64
// conversion runs per output block.
template <bool HAS_DF>
__global__ void __launch_bounds__(192) apply_factor_kernel(const ApplyJob* jobs,
                                                           const double2* __restrict__ work,
                                                           const float4* __restrict__ work_df,
                                                           const float4* __restrict__ scratch,
                                                           float2* out) {
    const ApplyJob J = jobs[blockIdx.x];
    const int row = threadIdx.x;
    if (row >= J.rows) return;
    const float4* T = scratch + J.t_off;
    constexpr int QB = 8;
    for (int q0 = 0; q0 < J.r; q0 += QB) {
        float acc[QB][4];  // (re_h, re_l, im_h, im_l)
#pragma unroll
        for (int q = 0; q < QB; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
        for (int p = 0; p < J.k; ++p) {
            float urh, uih, url, uil;
            if (HAS_DF) {
                const float4 u = work_df[J.src + row + (int64_t)p * J.src_ld];  // (re_h, im_h, re_l, im_l)
                urh = u.x;
                uih = u.y;
                url = u.z;
                uil = u.w;
            } else {
                const double2 ud = work[J.src + row + (int64_t)p * J.src_ld];
                urh = __double2float_rn(ud.x);
                uih = __double2float_rn(ud.y);
                url = __double2float_rn(ud.x - (double)urh);
                uil = __double2float_rn(ud.y - (double)uih);
            }
#pragma unroll
            for (int q = 0; q < QB; ++q)
                if (q0 + q < J.r) {
                    const float4 t = T[p + (int64_t)(q0 + q) * J.k];  // (re_h, im_h, re_l, im_l)
                    // re += u_re t_re - u_im t_im ; im += u_re t_im + u_im t_re
                    df_mac(acc[q][0], acc[q][1], urh, url, t.x, t.z);
                    df_mac(acc[q][0], acc[q][1], -uih, -uil, t.y, t.w);
                    df_mac(acc[q][2], acc[q][3], urh, url, t.y, t.w);
                    df_mac(acc[q][2], acc[q][3], uih, uil, t.x, t.z);
                }
        }
#pragma unroll
        for (int q = 0; q < QB; ++q)
            if (q0 + q < J.r)
                out[J.dst + row + (int64_t)(q0 + q) * J.ld] =
                    make_float2(__fadd_rn(acc[q][0], acc[q][1]), __fadd_rn(acc[q][2], acc[q][3]));
    }
}

}  // namespace

// ---- host drivers ----
struct RecompBatch {
    std::vector<CoreJob> jobs;
    CoreJob* d_jobs = nullptr;
    double2* d_scratch = nullptr;
    int32_t* d_rank = nullptr;
};

void* recompress_core(const std::vector<int64_t>& u_off, const std::vector<int64_t>& v_off,
                      const std::vector<int64_t>& m3, const std::vector<int64_t>& n3,
                      const std::vector<int32_t>& k, const std::vector<int64_t>& g_off,
                      const std::vector<int32_t>& g_ld, const double2* d_gram, int recompress,
                      double2* d_work, double eps, std::vector<int32_t>& ranks,
                      std::vector<int64_t>& s_off, cudaStream_t st) {
    RecompBatch* B = new RecompBatch();
    const size_t nj = k.size();
    B->jobs.resize(nj);
    s_off.resize(nj);
    int64_t off = 0;
    int kmax = 1;
    for (size_t j = 0; j < nj; ++j) {
        CoreJob& c = B->jobs[j];
        c.u_off = u_off[j];
        c.v_off = v_off[j];
        c.m3 = m3[j];
        c.n3 = n3[j];
        c.k = k[j];
        c.g_off = g_off[j];
        c.g_ld = g_ld[j];
        c.pad_ = 0;
        c.recompress = recompress;
        c.s_off = off;
        s_off[j] = off;
        off += 6 * (int64_t)k[j] * k[j];
        kmax = std::max(kmax, (int)k[j]);
    }
    if (kmax > 768) hm_throw(HM_ERR_UNSUPPORTED, "ACA rank above 768 columns");
    HM_CUDA(cudaMallocAsync((void**)&B->d_jobs, std::max<size_t>(nj, 1) * sizeof(CoreJob), st));
    HM_CUDA(cudaMallocAsync((void**)&B->d_scratch, std::max<int64_t>(off, 1) * sizeof(double2), st));
    HM_CUDA(cudaMallocAsync((void**)&B->d_rank, std::max<size_t>(nj, 1) * sizeof(int32_t), st));
    HM_CUDA(cudaMemcpyAsync(B->d_jobs, B->jobs.data(), nj * sizeof(CoreJob), cudaMemcpyHostToDevice, st));
    bool need_tile = false;
    for (size_t j = 0; j < nj; ++j) need_tile |= g_off[j] < 0;
    const size_t smem = need_tile ? (size_t)TILE_ROWS * kmax * sizeof(double2) : 0;
    // static (about 20 KB) + dynamic shared memory may exceed the 48 KB default
    HM_CUDA(cudaFuncSetAttribute(recomp_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    if (nj) {
        recomp_core_kernel<<<(unsigned)nj, RT, smem, st>>>(B->d_jobs, d_work, d_gram,
                                                          B->d_scratch, eps, B->d_rank, kmax);
                                                          HM_LAUNCHED();
        HM_CUDA(cudaGetLastError());
    }
    ranks.resize(nj);
    HM_CUDA(cudaMemcpyAsync(ranks.data(), B->d_rank, nj * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    return B;
}

// Applies T_U / T_V to the factors and writes the chunks.  items: for every
// (job, leaf) pair: (job, which: 0 = U / 1 = V, first row in the factor, rows,
// arena offset, ld).  d_work_df: the double-float copy of d_work (same
// offsets), or null.
void recompress_apply(void* batch, const std::vector<int64_t>& job_of,
                      const std::vector<int32_t>& which, const std::vector<int64_t>& row0,
                      const std::vector<int32_t>& rows, const std::vector<int64_t>& dst,
                      const std::vector<int32_t>& ld, const std::vector<int32_t>& ranks,
                      const double2* d_work, const float4* d_work_df, float2* d_out, cudaStream_t st) {
    RecompBatch* B = (RecompBatch*)batch;
    std::vector<ApplyJob> aj;
    aj.reserve(job_of.size());
    for (size_t i = 0; i < job_of.size(); ++i) {
        const CoreJob& c = B->jobs[job_of[i]];
        const int32_t r = ranks[job_of[i]];
        if (r == 0) continue;
        ApplyJob a;
        const int64_t k2 = (int64_t)c.k * c.k;
        if (which[i] == 0) {
            a.src = c.u_off + row0[i];
            a.src_ld = c.m3;
            a.t_off = c.s_off + 4 * k2;
        } else {
            a.src = c.v_off + row0[i];
            a.src_ld = c.n3;
            a.t_off = c.s_off + 5 * k2;
        }
        a.dst = dst[i];
        a.k = c.k;
        a.r = r;
        a.rows = rows[i];
        a.ld = ld[i];
        if (a.rows > 192) hm_throw(HM_ERR_ARG, "factor slice longer than 192 rows");
        aj.push_back(a);
    }
    if (!aj.empty()) {
        ApplyJob* d = nullptr;
        HM_CUDA(cudaMallocAsync((void**)&d, aj.size() * sizeof(ApplyJob), st));
        HM_CUDA(cudaMemcpyAsync(d, aj.data(), aj.size() * sizeof(ApplyJob), cudaMemcpyHostToDevice, st));
        if (d_work_df)
            apply_factor_kernel<true><<<(unsigned)aj.size(), 192, 0, st>>>(
                d, d_work, d_work_df, reinterpret_cast<const float4*>(B->d_scratch), d_out);
        else
            apply_factor_kernel<false><<<(unsigned)aj.size(), 192, 0, st>>>(
                d, d_work, nullptr, reinterpret_cast<const float4*>(B->d_scratch), d_out);
        HM_LAUNCHED();
        HM_CUDA(cudaGetLastError());
        HM_CUDA(cudaFreeAsync(d, st));
    }
}

void recompress_release(void* batch, cudaStream_t st) {
    RecompBatch* B = (RecompBatch*)batch;
    if (!B) return;
    if (B->d_jobs) HM_CUDA(cudaFreeAsync(B->d_jobs, st));
    if (B->d_scratch) HM_CUDA(cudaFreeAsync(B->d_scratch, st));
    if (B->d_rank) HM_CUDA(cudaFreeAsync(B->d_rank, st));
    delete B;
}

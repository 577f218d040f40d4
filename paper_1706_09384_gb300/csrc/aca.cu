// aca.cu — batched vector ACA (Sec. 2.2, partially pivoted ACA in six steps,
// with the rank-3 update and sigma_3 pivot of Sec. 2.3, strategy 3).
//
// One CTA compresses one admissible block at a time (persistent grid, dynamic
// queue).  Per step:
//   1. row block R(i^, :) = A(i^, :) - U(i^, :) V^H          (3 x 3n, FP64)
//   2. j^ = argmax over unused j of sigma_3(R(i^, j)); gamma = R(i^, j^)^{-1}
//      (a singular maximum, sigma_3 <= 1e-12 s_ref, retires row i^ and
//      restarts on the lowest unused row; s_ref = largest sigma_1 seen)
//   3. column block C = A(:, j^) - U V(j^, :)^H               (3m x 3)
//   4. next i^ = argmax over unused i of sigma_3(C(i, :)), on C before the update
//   5. U_{k+1} = C gamma, V_{k+1} = R(i^, :)^H
//   6. ||B_{k+1}||_F^2 = ||B_k||^2 + 2 Re <B_k, dB> + ||dB||^2, FP64
//   stop when ||dB||_F <= eps ||B_{k+1}||_F (Eq. stop_part read for rank 3),
//   when no row is left, or at full rank.  Ties in an argmax go to the lowest
//   index.  The factors live in a global workspace with a fixed column
//   capacity (double-float pairs in the build, FP64 in the allocation-free
//   entry point); a block that needs more reports an overflow and is re-run
//   with a larger capacity by the host.
//
// sigma_1 and sigma_3 of a 3x3 block M are computed from the invariants of
// M^H M: e1 = ||M||_F^2, e2 = sum of |2x2 minors|^2, e3 = |det M|^2 (the
// coefficients of its characteristic polynomial), whose roots follow from
// the trigonometric solution of the cubic; when the smallest root is below
// 1e-4 of the largest it is recomputed from the deflated quadratic
// (sum = (e2 - e3/l1)/l1, product = e3/l1), which keeps sigma_3 accurate to
// the precision of det M.
#include <algorithm>

#include "hm_internal.h"

namespace {

constexpr int AT = 256;             // threads of an ACA CTA
constexpr int ACA_MIN_CTAS = 2;     // resident CTAs per SM the launch bounds ask for
constexpr int AW = AT / 32;
constexpr int ACA_CH = 256;         // rows of the new factor columns staged per chunk (step 6)
constexpr double SING_REL = 1e-12;

// A complex value from lane `src` of the first nine lanes of warp 0.
HM_D double2 shfl9(double2 v, int src) {
    return make_double2(__shfl_sync(0x1ffu, v.x, src), __shfl_sync(0x1ffu, v.y, src));
}

HM_D double2 minor2(const double2 M[9], int r0, int r1, int c0, int c1) {
    return csub(cmul(M[3 * r0 + c0], M[3 * r1 + c1]), cmul(M[3 * r0 + c1], M[3 * r1 + c0]));
}

// sigma_1 and sigma_3 of a 3x3 complex block (cofactors streamed one at a time).
HM_D void sv13(const double2 M[9], double& s1, double& s3) {
    double e1 = 0.0, e2 = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) e1 += cabs2(M[q]);
    const double2 c0 = minor2(M, 1, 2, 1, 2);
    const double2 c1 = minor2(M, 1, 2, 0, 2);   // cofactor is -c1
    const double2 c2 = minor2(M, 1, 2, 0, 1);
    const double2 det = cadd(csub(cmul(M[0], c0), cmul(M[1], c1)), cmul(M[2], c2));
    e2 = cabs2(c0) + cabs2(c1) + cabs2(c2);
    e2 += cabs2(minor2(M, 0, 2, 1, 2)) + cabs2(minor2(M, 0, 2, 0, 2)) + cabs2(minor2(M, 0, 2, 0, 1));
    e2 += cabs2(minor2(M, 0, 1, 1, 2)) + cabs2(minor2(M, 0, 1, 0, 2)) + cabs2(minor2(M, 0, 1, 0, 1));
    const double e3 = cabs2(det);
    if (e1 == 0.0) {
        s1 = 0.0;
        s3 = 0.0;
        return;
    }
    const double mm = e1 / 3.0;
    const double p = fmax(mm * mm - e2 / 3.0, 0.0);
    double l1, l3;
    if (p <= 0.0) {
        l1 = mm;
        l3 = mm;
    } else {
        const double q = mm * mm * mm - 0.5 * mm * e2 + 0.5 * e3;
        const double sp = sqrt(p);
        const double cth = fmin(fmax(q / (p * sp), -1.0), 1.0);
        const double th = acos(cth) / 3.0;
        l1 = mm + 2.0 * sp * cos(th);
        l3 = mm + 2.0 * sp * cos(th + 2.0943951023931954923);
    }
    if (l3 < 1e-4 * l1) {  // deflate: the two small roots from the quadratic
        const double P = e3 / l1;
        const double s = (e2 - P) / l1;
        const double disc = fmax(s * s - 4.0 * P, 0.0);
        const double l2 = 0.5 * (s + sqrt(disc));
        l3 = l2 > 0.0 ? P / l2 : 0.0;
    }
    s1 = sqrt(fmax(l1, 0.0));
    s3 = sqrt(fmax(l3, 0.0));
}

// FP32 estimate of (sigma_1, sigma_3) used to shortlist pivot candidates.  The
// entries are truncated to FP32 on the integer pipes (a relative change below
// 2^-23, far inside the shortlist margin); the block is then scaled by its
// largest entry so that |det|^2 (~ sigma^6) stays in the normal FP32 range for
// small residuals or weighted entries.
HM_D void sv13f(const double2 Md[9], float& s1, float& s3) {
    float2 M[9];
    float amax = 0.f;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        M[q] = make_float2(f64_to_f32_rz_bits(Md[q].x), f64_to_f32_rz_bits(Md[q].y));
        amax = fmaxf(amax, fmaxf(fabsf(M[q].x), fabsf(M[q].y)));
    }
    if (!(amax > 0.f) || !(amax < 3.0e38f)) {  // zero, non-finite or NaN block
        s1 = s3 = (amax == 0.f) ? 0.f : __int_as_float(0x7fc00000);
        return;
    }
    const float isc = 1.f / amax;
#pragma unroll
    for (int q = 0; q < 9; ++q) M[q] = make_float2(M[q].x * isc, M[q].y * isc);
    auto mn = [&](int r0, int r1, int c0, int c1) {
        const float2 a = M[3 * r0 + c0], b = M[3 * r1 + c1], c = M[3 * r0 + c1], d = M[3 * r1 + c0];
        return make_float2(a.x * b.x - a.y * b.y - (c.x * d.x - c.y * d.y),
                           a.x * b.y + a.y * b.x - (c.x * d.y + c.y * d.x));
    };
    auto ab2 = [](float2 z) { return z.x * z.x + z.y * z.y; };
    float e1 = 0.f;
#pragma unroll
    for (int q = 0; q < 9; ++q) e1 += ab2(M[q]);
    const float2 c0 = mn(1, 2, 1, 2), c1 = mn(1, 2, 0, 2), c2 = mn(1, 2, 0, 1);
    const float2 det = make_float2(M[0].x * c0.x - M[0].y * c0.y - (M[1].x * c1.x - M[1].y * c1.y) +
                                       M[2].x * c2.x - M[2].y * c2.y,
                                   M[0].x * c0.y + M[0].y * c0.x - (M[1].x * c1.y + M[1].y * c1.x) +
                                       M[2].x * c2.y + M[2].y * c2.x);
    float e2 = ab2(c0) + ab2(c1) + ab2(c2) + ab2(mn(0, 2, 1, 2)) + ab2(mn(0, 2, 0, 2)) +
               ab2(mn(0, 2, 0, 1)) + ab2(mn(0, 1, 1, 2)) + ab2(mn(0, 1, 0, 2)) + ab2(mn(0, 1, 0, 1));
    const float e3 = ab2(det);
    if (!(e1 > 0.f)) {
        s1 = e1 == 0.f ? 0.f : e1;  // NaN propagates
        s3 = s1;
        return;
    }
    const float mm = e1 / 3.f;
    const float pp = fmaxf(mm * mm - e2 / 3.f, 0.f);
    float l1, l3;
    if (pp <= 0.f) {
        l1 = l3 = mm;
    } else {
        const float q = mm * mm * mm - 0.5f * mm * e2 + 0.5f * e3;
        const float sp = sqrtf(pp);
        const float th = acosf(fminf(fmaxf(q / (pp * sp), -1.f), 1.f)) / 3.f;
        l1 = mm + 2.f * sp * cosf(th);
        l3 = mm + 2.f * sp * cosf(th + 2.0943951f);
    }
    if (l3 < 1e-3f * l1) {
        const float P = e3 / l1;
        const float sm = (e2 - P) / l1;
        const float l2 = 0.5f * (sm + sqrtf(fmaxf(sm * sm - 4.f * P, 0.f)));
        l3 = l2 > 0.f ? P / l2 : 0.f;
    }
    s1 = sqrtf(fmaxf(l1, 0.f)) * amax;
    s3 = sqrtf(fmaxf(l3, 0.f)) * amax;
}

// A candidate whose FP32 sigma_3 is within this fraction of its sigma_1 of the
// best lower bound is re-evaluated in FP64.  The FP32 invariant formula errs by
// up to ~2.3e-3 sigma_1 (near-triple roots, measured over U and T blocks), so
// the margin keeps the FP64 argmax on the shortlist with room to spare.
constexpr float SHORTLIST_REL = 2e-2f;

struct BlockRed {
    double v[AW];
    int64_t i[AW];
    double w[AW];
};

// CTA argmax of (v, i) (ties -> lowest i) and max of w; result to all threads.
HM_D void block_argmax(double& v, int64_t& i, double& w, BlockRed& sh) {
    warp_argmax(v, i);
    for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh.v[wid] = v;
        sh.i[wid] = i;
        sh.w[wid] = w;
    }
    __syncthreads();
    v = sh.v[0];
    i = sh.i[0];
    w = sh.w[0];
    for (int q = 1; q < AW; ++q) {
        argmax_merge(v, i, sh.v[q], sh.i[q]);
        w = fmax(w, sh.w[q]);
    }
}

// Warp sum of N values with a halving exchange: at each level a lane keeps the
// half of its values that its partner does not, so each level costs half the
// shuffles and adds of the previous one (about 2N instead of 5N for N >= 32).
// On return every lane holds all N totals.
template <int N>
HM_D void warp_sum_many(double (&x)[N]) {
    const int lane = threadIdx.x & 31;
    if (N >= 4) {
        constexpr int H = N / 2;
        const bool up = (lane & 16) != 0;
        // level 1: lanes < 16 keep values [0, H), lanes >= 16 keep [H, N)
        double y[N - H > H ? N - H : H];
#pragma unroll
        for (int q = 0; q < (N - H > H ? N - H : H); ++q) {
            const int mine = up ? H + q : q, theirs = up ? q : H + q;
            const double send = (theirs < N && (up ? q < H : H + q < N)) ? x[theirs] : 0.0;
            const double got = __shfl_xor_sync(0xffffffffu, send, 16);
            y[q] = (mine < N ? x[mine] : 0.0) + got;
        }
        // levels 2..5 on the kept half (plain butterflies)
#pragma unroll
        for (int q = 0; q < (N - H > H ? N - H : H); ++q)
            for (int o = 8; o > 0; o >>= 1) y[q] += __shfl_xor_sync(0xffffffffu, y[q], o);
        // gather the two halves back to every lane
#pragma unroll
        for (int q = 0; q < (N - H > H ? N - H : H); ++q) {
            const double other = __shfl_xor_sync(0xffffffffu, y[q], 16);
            if (up) {
                if (q < H) x[q] = other;
                if (H + q < N) x[H + q] = y[q];
            } else {
                if (q < H) x[q] = y[q];
                if (H + q < N) x[H + q] = other;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) x[q] = warp_sum(x[q]);
    }
}

// ---- double-float residuals (FP32 pairs, ~44 significant bits) ----
// The residual rows and columns of steps 1 and 3 subtract sum_p U(i, p)
// conj(V(j, p)) from the Green's tensors: k complex multiply-adds per entry,
// the bulk of the ACA's arithmetic.  On GB300 FP64 runs at 1/64 of the FP32
// rate, so these sums run in double-float arithmetic (Dekker's product with an
// FMA, Knuth's two-sum; every operation an explicitly rounded intrinsic so
// nothing is fused) over U and V stored as double-float pairs (each new
// column formed in FP64, then split), and the difference with the FP64 tensor
// is taken in FP64.  The pivots and the norm updates of step 6 (sums rounded
// to FP64 once per thread) stay FP64.
__device__ __forceinline__ void dfm(float& h, float& l, float ah, float al, float bh, float bl) {
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
// s += u conj(v) for double-float complex u, v = (re_h, im_h, re_l, im_l)
__device__ __forceinline__ void df_cmac_conj(float (&s)[4], float4 u, float4 v) {
    dfm(s[0], s[1], u.x, u.z, v.x, v.z);    // re += ur vr
    dfm(s[0], s[1], u.y, u.w, v.y, v.w);    // re += ui vi
    dfm(s[2], s[3], u.y, u.w, v.x, v.z);    // im += ui vr
    dfm(s[2], s[3], -u.x, -u.z, v.y, v.w);  // im -= ur vi
}
// The double-float copy of an FP64 value: hi = v truncated to FP32, lo = the
// exact FP64 remainder truncated to FP32 (~46 significant bits in all), the
// conversions on the integer pipes.
__device__ __forceinline__ float4 df_of(double2 v) {
    const float rh = f64_to_f32_rz_bits(v.x), ih = f64_to_f32_rz_bits(v.y);
    return make_float4(rh, ih, f64_to_f32_rz_bits(v.x - f32_to_f64_bits(rh)),
                       f64_to_f32_rz_bits(v.y - f32_to_f64_bits(ih)));
}
// g -= s, the double-float sum subtracted in FP64 part by part (the parts
// converted on the integer pipes)
__device__ __forceinline__ void sub_df(double2& g, const float (&s)[4]) {
    g.x = (g.x - f32_to_f64_bits(s[0])) - f32_to_f64_bits(s[1]);
    g.y = (g.y - f32_to_f64_bits(s[2])) - f32_to_f64_bits(s[3]);
}

// Step 6 of the ACA, one side: out[q] = sum over the nr rows of x conj(new_q)
// (side 1, x = column p of V) or new_q conj(x) (side 0, x = column p of U),
// for the column p of this thread; threads tid = g P + pl (g < G), p = p0 + pl.  The
// three new columns (k, k + 1, k + 2 of base) are staged in shared memory
// ACA_CH rows at a time; group g sums its slice of each chunk in double-float
// arithmetic, the slices are rounded to FP64 once and added in FP64; out is
// set for g = 0.  Every thread of the CTA calls it (block barriers inside).
// Not inlined: it keeps the ACA kernel's register allocation out of the loop.
__device__ __noinline__ void df_cross_side(const float4* base, int64_t nr, int k, int p, int NP, int g, int G,
                                           int pl, int P, int side, float4 (*s_new)[ACA_CH],
                                           double2 (*s_red)[3], double2* out) {
    const int tid = threadIdx.x;
    float acc[3][4] = {};
    for (int64_t r0 = 0; r0 < nr; r0 += ACA_CH) {
        const int cn = (int)min((int64_t)ACA_CH, nr - r0);
        __syncthreads();  // the previous chunk is consumed
        for (int t = tid; t < 3 * cn; t += AT) {
            const int q = t / cn, rr = t - q * cn;
            s_new[q][rr] = base[(int64_t)(k + q) * nr + r0 + rr];
        }
        __syncthreads();
        if (p < NP && g < G) {
            const float4* col = base + (int64_t)p * nr + r0;
            const int rb = g * cn / G, re = (g + 1) * cn / G;
            auto mac = [&](const float4& x, int rr) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (side)
                        df_cmac_conj(acc[q], x, s_new[q][rr]);  // V_p conj(Vn_q)
                    else
                        df_cmac_conj(acc[q], s_new[q][rr], x);  // Un_q conj(U_p)
                }
            };
            int rr = rb;
            for (; rr + 1 < re; rr += 2) {  // two rows' loads in flight
                const float4 x0 = col[rr], x1 = col[rr + 1];
                mac(x0, rr);
                mac(x1, rr + 1);
            }
            if (rr < re) mac(col[rr], rr);
        }
    }
    if (g < G)
#pragma unroll
        for (int q = 0; q < 3; ++q)
            s_red[g * P + pl][q] =
                make_double2((double)acc[q][0] + (double)acc[q][1], (double)acc[q][2] + (double)acc[q][3]);
    __syncthreads();
    if (g == 0 && p < NP)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            double2 t2 = s_red[pl][q];
            for (int h = 1; h < G; ++h) t2 = cadd(t2, s_red[h * P + pl][q]);
            out[q] = t2;
        }
    __syncthreads();  // s_red is free again
}

template <int N>
HM_D void block_sum(double (&x)[N], double (*sh)[AW]) {
    warp_sum_many<N>(x);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < N; ++q) sh[q][wid] = x[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < N; ++q) {
        double s = 0.0;
        for (int w = 0; w < AW; ++w) s += sh[q][w];
        x[q] = s;
    }
}

template <bool DF>
__global__ void __launch_bounds__(AT, ACA_MIN_CTAS) aca_kernel(GreenParams gp0,
                                                 const GreenParams* __restrict__ gps,
                                                 const double* __restrict__ pts,
                                                 const double* __restrict__ nrm,
                                                 const AcaJob* __restrict__ jobs, int64_t njobs,
                                                 int* counter, double2* work, double2* gram,
                                                 unsigned char* flags, int64_t flag_stride,
                                                 double2* rowbuf, double2* colbuf,
                                                 int64_t rb_stride, int64_t cb_stride,
                                                 int capmax, double eps, AcaResult* res,
                                                 float4* work_df) {
    extern __shared__ double2 smem[];
    double2* Urow = smem;             // 3 x capmax: U(3 i^ + a, p)
    double2* Vrow = smem + 3 * capmax;  // 3 x capmax: V(3 j^ + c, p)
    // DF: the same rows as double-float pairs (same 16 bytes per entry)
    float4* Urow_df = reinterpret_cast<float4*>(smem);
    float4* Vrow_df = reinterpret_cast<float4*>(smem + 3 * capmax);
    __shared__ BlockRed red;
    __shared__ double sums[36][AW];
    __shared__ int64_t s_job, s_ihat, s_jhat, s_inext;
    __shared__ int s_k;
    __shared__ double s_normB2, s_sref, s_best, s_dB2;
    __shared__ double2 s_gam[9];
    __shared__ double2 s_gdu[9], s_gdv[9];  // new diagonal Gram blocks (double-float path)
    __shared__ float4 s_new[3][ACA_CH];       // step 6: a chunk of the three new columns
    __shared__ double2 s_red[AT][3];          // step 6: partial sums of the thread groups
    __shared__ int s_stop;   // 0 continue, 1 converged, 2 overflow, 3 non-finite
    __shared__ int s_lost;   // a row retired for singular pivots carried a non-negligible residual
    __shared__ GreenParams s_gp;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double2* R = rowbuf + blockIdx.x * rb_stride;   // [a][3n], row-major, then n float2
    double2* C = colbuf + blockIdx.x * cb_stride;   // [3m][3], row-major, then m float2
    unsigned char* used = flags + blockIdx.x * flag_stride;

    for (;;) {
        if (tid == 0) s_job = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t job = s_job;
        if (job >= njobs) return;
        const AcaJob J = jobs[job];
        // one problem (kernel parameters), or a batch of problems (J.pad_ =
        // problem index; its parameters are read from shared memory)
        if (gps && tid == 0) s_gp = gps[J.pad_];
        const GreenParams& gp = gps ? s_gp : gp0;
        const int64_t m = J.m, n = J.n, m3 = 3 * m, n3 = 3 * n;
        // DF: the factors are kept only as double-float pairs (every later
        // reader, the residuals, the norm update and the factor application,
        // takes those), the FP64 path keeps them in FP64
        double2* U = DF ? nullptr : work + J.u_off;
        double2* V = DF ? nullptr : work + J.v_off;
        float4* Ud = DF ? work_df + J.u_off : nullptr;
        float4* Vd = DF ? work_df + J.v_off : nullptr;
        double2* GU = (gram && J.g_off >= 0) ? gram + J.g_off : nullptr;  // U^H U, ld cap
        double2* GV = GU ? GU + (int64_t)J.cap * J.cap : nullptr;          // V^H V, ld cap
        unsigned char* urow = used;
        unsigned char* ucol = used + m;
        for (int64_t q = tid; q < m + n; q += AT) used[q] = 0;
        if (tid == 0) {
            s_k = 0;
            s_ihat = 0;
            s_normB2 = 0.0;
            s_sref = 0.0;
            s_stop = 0;
            s_lost = 0;
        }
        const int64_t steps_max = m < n ? m : n;
        float2* Rs = reinterpret_cast<float2*>(R + 9 * n);  // FP32 (sigma_1, sigma_3) of row candidates
        float2* Cs = reinterpret_cast<float2*>(C + 9 * m);  // ... of column candidates
        const double* xr = pts + 3 * J.tau_begin;
        const double* xc = pts + 3 * J.sig_begin;
        const double* nc = nrm ? nrm + 3 * J.sig_begin : nullptr;
        __syncthreads();

        while (s_stop == 0) {
            const int k = s_k;
            const int64_t ihat = s_ihat;
            for (int t = tid; t < 3 * k; t += AT) {
                const int a = t / k, p = t - a * k;
                if (DF)
                    Urow_df[a * capmax + p] = Ud[3 * ihat + a + (int64_t)p * m3];
                else
                    Urow[a * capmax + p] = U[3 * ihat + a + (int64_t)p * m3];
            }
            __syncthreads();
            // ---- step 1-2: row residual and sigma_3 pivot search ----
            float bestf = -1.f, s1maxf = 0.f;  // the shortlist's bounds in FP32
            int64_t bj = -1;
            for (int64_t j = tid; j < n; j += AT) {
                // the double-float sums first, the FP64 tensor after them: G is not
                // live across the loop (36 registers)
                float s9[9][4] = {};
                if (DF && k > 0) {
                    // V(j, p) for p + 1 is loaded while p is summed
                    const float4* vp = Vd + 3 * j;
                    float4 v0 = vp[0], v1 = vp[1], v2 = vp[2];
                    for (int p = 0; p < k; ++p) {
                        float4 w0 = v0, w1 = v1, w2 = v2;
                        if (p + 1 < k) {
                            const float4* vq = vp + (int64_t)(p + 1) * n3;
                            w0 = vq[0];
                            w1 = vq[1];
                            w2 = vq[2];
                        }
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float4 u = Urow_df[a * capmax + p];
                            df_cmac_conj(s9[3 * a + 0], u, v0);
                            df_cmac_conj(s9[3 * a + 1], u, v1);
                            df_cmac_conj(s9[3 * a + 2], u, v2);
                        }
                        v0 = w0;
                        v1 = w1;
                        v2 = w2;
                    }
                }
                double2 G[9];
                if (J.tau_begin + ihat == J.sig_begin + j) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) G[q] = make_double2((q % 4 == 0) ? gp.diag : 0.0, 0.0);
                } else {
                    green_tensor(gp, xr + 3 * ihat, xc + 3 * j, nc ? nc + 3 * j : nullptr, G);
                    apply_weight(gp, J.sig_begin + j, G);
                }
                if (DF && k > 0) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) sub_df(G[q], s9[q]);
                } else if (!DF) {
                    for (int p = 0; p < k; ++p) {
                        const double2* vp = V + (int64_t)p * n3 + 3 * j;
                        const double2 v0 = vp[0], v1 = vp[1], v2 = vp[2];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const double2 u = Urow[a * capmax + p];
                            cfms_conj(G[3 * a + 0], u, v0);
                            cfms_conj(G[3 * a + 1], u, v1);
                            cfms_conj(G[3 * a + 2], u, v2);
                        }
                    }
                }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int c = 0; c < 3; ++c) R[a * n3 + 3 * j + c] = G[3 * a + c];
                float s1f, s3f;
                sv13f(G, s1f, s3f);
                Rs[j] = make_float2(s1f, s3f);
                s1maxf = fmaxf(s1maxf, s1f);
                if (!ucol[j]) {
                    const float lo = s3f - SHORTLIST_REL * s1f;
                    if (lo > bestf || (bj < 0 && lo == lo)) {
                        bestf = lo;
                        bj = j;
                    }
                }
            }
            double best = bestf, s1max = s1maxf;
            block_argmax(best, bj, s1max, red);  // best = largest lower bound
            {
                // FP64 sigma_3 on the shortlist; exact argmax with ties to the lowest j
                const float lstar = (float)best;  // an FP32 value (exact)
                double b64 = -1.0, dummy = 0.0;
                int64_t j64 = -1;
                for (int64_t j = tid; j < n; j += AT) {
                    if (ucol[j]) continue;
                    const float2 sf = Rs[j];
                    if (!(sf.y + SHORTLIST_REL * sf.x >= lstar)) continue;
                    double2 G[9];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int c = 0; c < 3; ++c) G[3 * a + c] = R[a * n3 + 3 * j + c];
                    double s1, s3;
                    sv13(G, s1, s3);
                    argmax_merge(b64, j64, s3, j);
                }
                block_argmax(b64, j64, dummy, red);
                best = b64;
                bj = j64;
            }
            if (tid == 0) {
                s_sref = fmax(s_sref, s1max);
                s_jhat = bj;
                s_best = best;
            }
            __syncthreads();
            if (s_jhat < 0) {  // no comparable candidate: columns remain, so values were NaN
                if (tid == 0) s_stop = (k / 3 < steps_max) ? 3 : 1;
                __syncthreads();
                break;
            }
            if (!(s_best > SING_REL * s_sref)) {
                // singular pivot: retire row i^, restart on the lowest unused row;
                // a row with a non-negligible residual is lost to the approximation
                if (tid == 0) {
                    urow[ihat] = 1;
                    if (s1max > eps * s_sref) s_lost = 1;
                }
                __syncthreads();
                double v = -1.0, dummy = 0.0;
                int64_t li = -1;
                for (int64_t i = tid; i < m; i += AT)
                    if (!urow[i]) {
                        argmax_merge(v, li, 0.0, i);
                        break;
                    }
                block_argmax(v, li, dummy, red);
                if (tid == 0) {
                    if (li < 0 || !(s_best == s_best))
                        s_stop = (s_best == s_best) ? 1 : 3;
                    else
                        s_ihat = li;
                }
                __syncthreads();
                continue;
            }
            const int64_t jhat = s_jhat;
            if (tid < 9) {
                // gamma = R(i^, j^)^-1 = adj / det (adj = cofactor^T): lane q < 9
                // forms cofactor q, then the inverse entry q from cofactor 3 c + a
                const int q = tid, r = q / 3, c = q % 3;
                const int r0 = r == 0 ? 1 : 0, r1 = r == 2 ? 1 : 2;
                const int c0 = c == 0 ? 1 : 0, c1 = c == 2 ? 1 : 2;
                auto P = [&](int a, int b) { return R[a * n3 + 3 * jhat + b]; };
                double2 cof = csub(cmul(P(r0, c0), P(r1, c1)), cmul(P(r0, c1), P(r1, c0)));
                if ((r + c) & 1) cof = cscale(cof, -1.0);
                const double2 det = cadd(cadd(cmul(P(0, 0), shfl9(cof, 0)), cmul(P(0, 1), shfl9(cof, 1))),
                                         cmul(P(0, 2), shfl9(cof, 2)));
                s_gam[q] = cdiv(shfl9(cof, 3 * c + r), det);
                if (q == 0) {
                    urow[ihat] = 1;
                    ucol[jhat] = 1;
                }
            }
            for (int t = tid; t < 3 * k; t += AT) {
                const int c = t / k, p = t - c * k;
                if (DF)
                    Vrow_df[c * capmax + p] = Vd[3 * jhat + c + (int64_t)p * n3];
                else
                    Vrow[c * capmax + p] = V[3 * jhat + c + (int64_t)p * n3];
            }
            __syncthreads();
            // ---- step 3-4: column residual and next row ----
            float bestrf = -1.f;
            double unused = 0.0;
            int64_t bi = -1;
            for (int64_t i = tid; i < m; i += AT) {
                float s9[9][4] = {};  // double-float sums, then the FP64 tensor
                if (DF && k > 0) {
                    // U(i, p) for p + 1 is loaded while p is summed
                    const float4* up = Ud + 3 * i;
                    float4 u0 = up[0], u1 = up[1], u2 = up[2];
                    for (int p = 0; p < k; ++p) {
                        float4 w0 = u0, w1 = u1, w2 = u2;
                        if (p + 1 < k) {
                            const float4* uq = up + (int64_t)(p + 1) * m3;
                            w0 = uq[0];
                            w1 = uq[1];
                            w2 = uq[2];
                        }
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float4 v = Vrow_df[c * capmax + p];
                            df_cmac_conj(s9[0 + c], u0, v);
                            df_cmac_conj(s9[3 + c], u1, v);
                            df_cmac_conj(s9[6 + c], u2, v);
                        }
                        u0 = w0;
                        u1 = w1;
                        u2 = w2;
                    }
                }
                double2 G[9];
                if (J.tau_begin + i == J.sig_begin + jhat) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) G[q] = make_double2((q % 4 == 0) ? gp.diag : 0.0, 0.0);
                } else {
                    green_tensor(gp, xr + 3 * i, xc + 3 * jhat, nc ? nc + 3 * jhat : nullptr, G);
                    apply_weight(gp, J.sig_begin + jhat, G);
                }
                if (DF && k > 0) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) sub_df(G[q], s9[q]);
                } else if (!DF) {
                    for (int p = 0; p < k; ++p) {
                        const double2* up = U + (int64_t)p * m3 + 3 * i;
                        const double2 u0 = up[0], u1 = up[1], u2 = up[2];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const double2 v = Vrow[c * capmax + p];
                            cfms_conj(G[0 + c], u0, v);
                            cfms_conj(G[3 + c], u1, v);
                            cfms_conj(G[6 + c], u2, v);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) C[9 * i + q] = G[q];
                if (!urow[i]) {
                    float s1f, s3f;
                    sv13f(G, s1f, s3f);
                    Cs[i] = make_float2(s1f, s3f);
                    const float lo = s3f - SHORTLIST_REL * s1f;
                    if (lo > bestrf || (bi < 0 && lo == lo)) {
                        bestrf = lo;
                        bi = i;
                    }
                }
            }
            double bestr = bestrf;
            block_argmax(bestr, bi, unused, red);
            {
                const float lstar = (float)bestr;
                double b64 = -1.0;
                int64_t i64 = -1;
                for (int64_t i = tid; i < m; i += AT) {
                    if (urow[i]) continue;
                    const float2 sf = Cs[i];
                    if (!(sf.y + SHORTLIST_REL * sf.x >= lstar)) continue;
                    double2 G[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) G[q] = C[9 * i + q];
                    double s1, s3;
                    sv13(G, s1, s3);
                    argmax_merge(b64, i64, s3, i);
                }
                block_argmax(b64, i64, unused, red);
                bestr = b64;
                bi = i64;
            }
            if (tid == 0) s_inext = bi;
            if constexpr (DF) {
                // ---- step 5: new factor columns, formed in FP64, stored as double-float pairs ----
                if (k + 3 <= J.cap) {
                    for (int64_t r = tid; r < m3; r += AT)
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
                            for (int a = 0; a < 3; ++a) cfma(acc, C[3 * r + a], s_gam[3 * a + q]);
                            Ud[r + (int64_t)(k + q) * m3] = df_of(acc);
                        }
                    for (int64_t c = tid; c < n3; c += AT)
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            Vd[c + (int64_t)(k + a) * n3] = df_of(cconj(R[a * n3 + c]));
                }
                __syncthreads();  // publishes the new columns to the CTA
                if (k + 3 > J.cap) {
                    if (tid == 0) s_stop = 2;
                    __syncthreads();
                    break;
                }
                // ---- step 6: cross terms (U_p^H Un_q)(Vn_q^H V_p) of <B_k, dB> for p < k and the
                // new diagonal Gram blocks (p = k .. k + 2), as double-float dot products over the
                // double-float copies (FP32 pipes).  A small GEMM: each thread owns one column p
                // (P of them per pass), groups of threads split the rows, the three new columns
                // are staged in shared memory chunk by chunk, so every old column is read once;
                // each thread's partial sum is rounded to FP64 once and the groups add in FP64 ----
                double cre = 0.0, cim = 0.0;
                {
                    // P = k + 3 columns per pass (at most AT), G = AT / P row groups;
                    // threads g >= G only help to stage the chunks
                    const int NP = k + 3;
                    const int P = NP < AT ? NP : AT;
                    const int G = AT / P, pl = tid % P, g = tid / P;
                    for (int p0 = 0; p0 < NP; p0 += P) {
                        const int p = p0 + pl;
                        double2 xs[3], ys[3];
                        df_cross_side(Ud, m3, k, p, NP, g, G, pl, P, 0, s_new, s_red, xs);
                        df_cross_side(Vd, n3, k, p, NP, g, G, pl, P, 1, s_new, s_red, ys);
                        if (g == 0 && p < NP) {
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const double2 xq = xs[q];  // U_p^H Un_q
                                const double2 yq = ys[q];  // Vn_q^H V_p
                                if (p < k) {
                                    const double2 z = cmul(xq, yq);
                                    cre += z.x;
                                    cim += z.y;
                                    if (GU) {  // the new Gram columns, by Hermitian symmetry
                                        GU[p + (int64_t)(k + q) * J.cap] = xq;
                                        GU[(k + q) + (int64_t)p * J.cap] = cconj(xq);
                                        GV[(k + q) + (int64_t)p * J.cap] = yq;
                                        GV[p + (int64_t)(k + q) * J.cap] = cconj(yq);
                                    }
                                } else {
                                    s_gdu[3 * (p - k) + q] = xq;  // Un_{p-k}^H Un_q
                                    s_gdv[3 * q + (p - k)] = yq;  // Vn_q^H Vn_{p-k}
                                }
                            }
                        }
                    }
                }
                double cr[2] = {cre, cim};
                block_sum<2>(cr, sums);  // its barriers also publish s_gdu, s_gdv
                if (tid == 0) {
                    // ||dB||^2 = sum_{q,q2} (Un_q^H Un_q2)(Vn_q2^H Vn_q)
                    double dB2 = 0.0;
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int q2 = 0; q2 < 3; ++q2) dB2 += cmul(s_gdu[3 * q + q2], s_gdv[3 * q2 + q]).x;
                    if (GU) {
#pragma unroll
                        for (int q = 0; q < 3; ++q)
#pragma unroll
                            for (int q2 = 0; q2 < 3; ++q2) {
                                const int64_t at = (k + q) + (int64_t)(k + q2) * J.cap;
                                GU[at] = s_gdu[3 * q + q2];
                                GV[at] = s_gdv[3 * q + q2];
                            }
                    }
                    const double nb2 = s_normB2 + 2.0 * cr[0] + dB2;
                    s_normB2 = nb2;
                    const int k2 = k + 3;
                    s_k = k2;
                    if (!(nb2 == nb2) || !(dB2 == dB2))
                        s_stop = 3;
                    else if (sqrt(dB2) <= eps * sqrt(fmax(nb2, 0.0)))
                        s_stop = 1;
                    else if (s_inext < 0 || k2 / 3 >= steps_max)
                        s_stop = 1;
                    else
                        s_ihat = s_inext;
                }
                __syncthreads();
            } else {
            // ---- step 5: new factor columns and their Gram matrices ----
            double g[36];
#pragma unroll
            for (int q = 0; q < 36; ++q) g[q] = 0.0;
            if (k + 3 <= J.cap) {
                for (int64_t r = tid; r < m3; r += AT) {
                    double2 un[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
                        for (int a = 0; a < 3; ++a) cfma(acc, C[3 * r + a], s_gam[3 * a + q]);
                        un[q] = acc;
                        U[r + (int64_t)(k + q) * m3] = acc;
                        if (DF) Ud[r + (int64_t)(k + q) * m3] = df_of(acc);
                    }
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int q2 = 0; q2 < 3; ++q2) {
                            double2 z = make_double2(g[2 * (3 * q + q2)], g[2 * (3 * q + q2) + 1]);
                            cfma_conja(z, un[q], un[q2]);
                            g[2 * (3 * q + q2)] = z.x;
                            g[2 * (3 * q + q2) + 1] = z.y;
                        }
                }
                for (int64_t c = tid; c < n3; c += AT) {
                    double2 vn[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        vn[a] = cconj(R[a * n3 + c]);
                        V[c + (int64_t)(k + a) * n3] = vn[a];
                        if (DF) Vd[c + (int64_t)(k + a) * n3] = df_of(vn[a]);
                    }
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int q2 = 0; q2 < 3; ++q2) {
                            double2 z = make_double2(g[18 + 2 * (3 * q + q2)], g[18 + 2 * (3 * q + q2) + 1]);
                            cfma_conja(z, vn[q], vn[q2]);
                            g[18 + 2 * (3 * q + q2)] = z.x;
                            g[18 + 2 * (3 * q + q2) + 1] = z.y;
                        }
                }
            }
            block_sum<36>(g, sums);  // includes the barrier that publishes U, V
            if (tid == 0) {
                // ||dB||^2 = sum_{q,q'} (Un_q^H Un_q')(Vn_q'^H Vn_q)
                double dB2 = 0.0;
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int q2 = 0; q2 < 3; ++q2) {
                        const double2 gu = make_double2(g[2 * (3 * q + q2)], g[2 * (3 * q + q2) + 1]);
                        const double2 gv =
                            make_double2(g[18 + 2 * (3 * q2 + q)], g[18 + 2 * (3 * q2 + q) + 1]);
                        dB2 += cmul(gu, gv).x;
                    }
                s_dB2 = dB2;
                if (GU && k + 3 <= J.cap) {
                    // new diagonal blocks of the Gram matrices: Un^H Un and Vn^H Vn
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int q2 = 0; q2 < 3; ++q2) {
                            const int64_t at = (k + q) + (int64_t)(k + q2) * J.cap;
                            GU[at] = make_double2(g[2 * (3 * q + q2)], g[2 * (3 * q + q2) + 1]);
                            GV[at] = make_double2(g[18 + 2 * (3 * q + q2)], g[18 + 2 * (3 * q + q2) + 1]);
                        }
                }
            }
            if (k + 3 > J.cap) {
                if (tid == 0) s_stop = 2;
                __syncthreads();
                break;
            }
            // ---- step 6: cross term <B_k, dB> = sum_{p,q} (U_p^H Un_q)(Vn_q^H V_p) ----
            double cre = 0.0, cim = 0.0;
            for (int p = wid; p < k; p += AW) {
                double2 ax[3] = {}, ay[3] = {};
                const double2* Up = U + (int64_t)p * m3;
                const double2* Vp = V + (int64_t)p * n3;
                for (int64_t r = lane; r < m3; r += 32) {
                    const double2 u = Up[r];
#pragma unroll
                    for (int q = 0; q < 3; ++q) cfma_conja(ax[q], u, U[r + (int64_t)(k + q) * m3]);
                }
                for (int64_t c = lane; c < n3; c += 32) {
                    const double2 v = Vp[c];
#pragma unroll
                    for (int q = 0; q < 3; ++q) cfma_conja(ay[q], V[c + (int64_t)(k + q) * n3], v);
                }
                double xy[12];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    xy[2 * q] = ax[q].x;
                    xy[2 * q + 1] = ax[q].y;
                    xy[6 + 2 * q] = ay[q].x;
                    xy[6 + 2 * q + 1] = ay[q].y;
                }
                warp_sum_many<12>(xy);
                double x[6], y[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    x[q] = xy[q];
                    y[q] = xy[6 + q];
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const double2 xq = make_double2(x[2 * q], x[2 * q + 1]);  // U_p^H Un_q
                    const double2 yq = make_double2(y[2 * q], y[2 * q + 1]);  // Vn_q^H V_p
                    const double2 z = cmul(xq, yq);
                    cre += z.x;
                    cim += z.y;
                    if (GU && lane == 0) {  // the new Gram columns, by Hermitian symmetry
                        GU[p + (int64_t)(k + q) * J.cap] = xq;
                        GU[(k + q) + (int64_t)p * J.cap] = cconj(xq);
                        GV[(k + q) + (int64_t)p * J.cap] = yq;
                        GV[p + (int64_t)(k + q) * J.cap] = cconj(yq);
                    }
                }
            }
            double cr[2] = {lane == 0 ? cre : 0.0, lane == 0 ? cim : 0.0};
            block_sum<2>(cr, sums);
            if (tid == 0) {
                const double dB2 = s_dB2;
                const double nb2 = s_normB2 + 2.0 * cr[0] + dB2;
                s_normB2 = nb2;
                const int k2 = k + 3;
                s_k = k2;
                if (!(nb2 == nb2) || !(dB2 == dB2))
                    s_stop = 3;
                else if (sqrt(dB2) <= eps * sqrt(fmax(nb2, 0.0)))
                    s_stop = 1;
                else if (s_inext < 0 || k2 / 3 >= steps_max)
                    s_stop = 1;
                else
                    s_ihat = s_inext;
            }
            __syncthreads();
            }  // FP64 path
        }
        if (tid == 0) {
            res[job].k = s_k;
            res[job].status = s_stop == 1 ? (s_lost ? 3 : 0) : (s_stop == 2 ? 1 : 2);
        }
        __syncthreads();
    }
}

}  // namespace

void launch_aca(const GreenParams& gp, const double* d_pts_p, const double* d_nrm_p,
                const AcaJob* d_jobs, int64_t njobs, double2* d_work, double2* d_gram,
                unsigned char* d_flags,
                int64_t flag_stride, double2* d_rowbuf, double2* d_colbuf, int64_t rowbuf_stride,
                int64_t colbuf_stride, double eps, AcaResult* d_res, int nctas, int capmax,
                int* d_counter, cudaStream_t st, const GreenParams* d_gps, float4* d_work_df) {
    if (njobs == 0) return;
    const size_t smem = (size_t)6 * capmax * sizeof(double2);
    HM_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(int), st));
    if (d_work_df) {
        HM_CUDA(cudaFuncSetAttribute(aca_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        aca_kernel<true><<<nctas, AT, smem, st>>>(gp, d_gps, d_pts_p, d_nrm_p, d_jobs, njobs, d_counter,
                                                  d_work, d_gram, d_flags, flag_stride, d_rowbuf, d_colbuf,
                                                  rowbuf_stride, colbuf_stride, capmax, eps, d_res,
                                                  d_work_df);
    } else {
        HM_CUDA(cudaFuncSetAttribute(aca_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        aca_kernel<false><<<nctas, AT, smem, st>>>(gp, d_gps, d_pts_p, d_nrm_p, d_jobs, njobs, d_counter,
                                                   d_work, d_gram, d_flags, flag_stride, d_rowbuf,
                                                   d_colbuf, rowbuf_stride, colbuf_stride, capmax, eps,
                                                   d_res, nullptr);
    }
    HM_LAUNCHED();
    HM_CUDA(cudaGetLastError());
}

int aca_ctas_per_sm(int capmax) {
    int nb = 0;
    const size_t smem = (size_t)6 * capmax * sizeof(double2);
    HM_CUDA(cudaFuncSetAttribute(aca_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, aca_kernel<true>, AT, smem));
    return nb > 0 ? nb : 1;
}

// ---------------------------------------------------------------------------
// Allocation-free single-block ACA.  The paper has no counterpart; this entry
// point serves callers that may not call cudaMalloc (see include/hm.h).  All
// scratch of the ACA kernel for one block (points, normals, residual row and
// column buffers, row/column flags, job, result, queue counter) lives in one
// file-scope device array sized for blocks of up to HM_NOALLOC_MAX_POINTS
// points per side.  Host code must not use the array's name as a device
// address: its device address is taken with cudaGetSymbolAddress once per
// device, with that device current.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int64_t NA_MAXP = HM_NOALLOC_MAX_POINTS;
constexpr size_t na_align(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t NA_PTS = 0;                                        // [x; y], 3 doubles per point
constexpr size_t NA_NRM = NA_PTS + na_align(24 * 2 * NA_MAXP);      // normals at y in the same layout
constexpr size_t NA_ROW = NA_NRM + na_align(24 * 2 * NA_MAXP);      // 9 n complex128
constexpr size_t NA_COL = NA_ROW + na_align(16 * (9 * NA_MAXP + NA_MAXP / 2 + 1));  // 9 m complex128 + m float2
constexpr size_t NA_FLG = NA_COL + na_align(16 * (9 * NA_MAXP + NA_MAXP / 2 + 1));  // m + n bytes
constexpr size_t NA_JOB = NA_FLG + na_align(2 * NA_MAXP);
constexpr size_t NA_RES = NA_JOB + na_align(sizeof(AcaJob));
constexpr size_t NA_CNT = NA_RES + na_align(sizeof(AcaResult));
constexpr size_t NA_BYTES = NA_CNT + na_align(sizeof(int));

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
unsigned char* g_na_addr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set up on first use).
unsigned char* noalloc_scratch(int dev) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) hm_throw(HM_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        HM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_na_addr[dev] = (unsigned char*)p;
    }
    return g_na_addr[dev];
}

}  // namespace

extern "C" hm_status hm_aca_block_noalloc(int32_t kernel, double rho, double lambda, double mu,
                                          double omega, const double* x, int64_t m,
                                          const double* y, const double* ny, int64_t n,
                                          double eps, int32_t cap, void* uv, int32_t* rank,
                                          void* stream) {
    try {
        if (rank) *rank = -1;
        if (!x || !y || !uv || !rank) hm_throw(HM_ERR_ARG, "null pointer");
        if (m < 1 || n < 1 || m > NA_MAXP || n > NA_MAXP)
            hm_throw(HM_ERR_ARG, "block sides must hold 1.." + std::to_string(NA_MAXP) +
                                     " points (allocation-free scratch limit)");
        if (cap < 3 || cap > 768 || cap % 3) hm_throw(HM_ERR_ARG, "cap must be a multiple of 3 in 3..768");
        if (kernel != HM_KERNEL_U && kernel != HM_KERNEL_T) hm_throw(HM_ERR_ARG, "unknown kernel");
        if (kernel == HM_KERNEL_T && !ny) hm_throw(HM_ERR_ARG, "the T kernel needs normals");
        if (!(rho > 0) || !(mu > 0) || !(omega > 0) || !(lambda + 2 * mu > 0))
            hm_throw(HM_ERR_ARG, "bad material parameters");
        if (!(eps > 0 && eps < 1)) hm_throw(HM_ERR_ARG, "eps must lie in (0, 1)");
        if (reinterpret_cast<uintptr_t>(uv) % 16) hm_throw(HM_ERR_ARG, "uv must be 16-byte aligned");
        cudaStream_t st = (cudaStream_t)stream;
        int dev = 0;
        HM_CUDA(cudaGetDevice(&dev));
        unsigned char* base = noalloc_scratch(dev);
        double* pts = (double*)(base + NA_PTS);
        double* nrm = (double*)(base + NA_NRM);
        HM_CUDA(cudaMemcpyAsync(pts, x, 24 * m, cudaMemcpyDeviceToDevice, st));
        HM_CUDA(cudaMemcpyAsync(pts + 3 * m, y, 24 * n, cudaMemcpyDeviceToDevice, st));
        if (kernel == HM_KERNEL_T)
            HM_CUDA(cudaMemcpyAsync(nrm + 3 * m, ny, 24 * n, cudaMemcpyDeviceToDevice, st));
        AcaJob J;
        J.tau_begin = 0;
        J.m = m;
        J.sig_begin = m;
        J.n = n;
        J.u_off = 0;
        J.v_off = 3 * m * (int64_t)cap;
        J.g_off = -1;
        J.cap = cap;
        J.pad_ = 0;
        AcaJob* d_job = (AcaJob*)(base + NA_JOB);
        AcaResult* d_res = (AcaResult*)(base + NA_RES);
        HM_CUDA(cudaMemcpyAsync(d_job, &J, sizeof(J), cudaMemcpyHostToDevice, st));
        const GreenParams gp = make_green_params(kernel, rho, lambda, mu, omega, 1.0);
        launch_aca(gp, pts, kernel == HM_KERNEL_T ? nrm : nullptr, d_job, 1, (double2*)uv, nullptr,
                   base + NA_FLG, m + n, (double2*)(base + NA_ROW), (double2*)(base + NA_COL),
                   9 * n + n / 2 + 1, 9 * m + m / 2 + 1, eps, d_res, 1, cap, (int*)(base + NA_CNT), st);
        AcaResult R;
        HM_CUDA(cudaMemcpyAsync(&R, d_res, sizeof(R), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        if (R.status == 1) hm_throw(HM_ERR_ARG, "ACA rank exceeds cap; call again with a larger cap");
        if (R.status == 2) hm_throw(HM_ERR_NUMERIC, "non-finite value in the ACA");
        if (R.status == 3)
            hm_throw(HM_ERR_UNSUPPORTED,
                     "rows with singular 3x3 blocks only: the vector ACA cannot pivot them "
                     "(store the block dense)");
        *rank = R.k;
    } catch (const hm_error& e) {
        hm_set_error(e.msg);
        return e.st;
    } catch (...) {
        hm_set_error("unexpected internal error");
        return HM_ERR_CUDA;
    }
    return HM_OK;
}

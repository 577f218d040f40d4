// matvec.cu — H-matrix-vector product y = A_H x (Sec. 3.1): dense product on
// the non-admissible leaves, U (V^H x) on the admissible ones.
//
// Storage layout ("chunk-major"): every block is cut along the storage
// segments of its row set (dense blocks, U factors) or column set (V factors):
// the leaf clusters, a leaf above 64 points cut into contiguous ranges of at
// most 64 points.  A chunk is a column-major (ld x ncols) complex matrix,
// ld = 3|segment| rounded up to an even count so each column starts on a
// 16-byte boundary.  All chunks that feed the rows of one segment are stored
// back to back, so the product streams the arena once, front to back.
//
// Phase 1:  t_b = V_b^H x_sigma     (per column segment; partial sums by atomics)
// Phase 2:  y_l = sum D x_sigma + sum U_b t_b   (per row segment)
// Both phases are HBM-bound (one complex FMA per stored complex entry).
// Work items are slices of a segment's chunk list of bounded byte size, so the
// grid load-balances; each CTA keeps partial sums per warp in registers and
// reduces them once.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "matvec_dev.cuh"
#include "pipeline.cuh"

namespace {

constexpr int MV_THREADS = 256;
constexpr int MV_WARPS = MV_THREADS / 32;
constexpr int PAIRS_PER_LANE = MAX_LD / 64;  // row pairs per lane (3)

__device__ __forceinline__ float4 ldg_stream(const float4* p) { return __ldcs(p); }

// Types of the fast product (x, t, y and the sums in FP32); the accurate
// product of the GMRES restarts has its own double-float kernels below.
template <bool ACC> struct MvT;
template <> struct MvT<false> {
    using R = float;
    using C2 = float2;
    struct C4 { float x, y, z, w; };
};

__device__ __forceinline__ float red_sum(float v) { return warp_sumf(v); }
// *p += (re, im) as a reduction (no value returned, so no round trip to wait for)
__device__ __forceinline__ void atomic_add_c(float2* p, float re, float im) {
    asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(re), "f"(im) : "memory");
}

// Phase 1: for every V chunk of the item's column leaf, t[vec + c] += V[:, c]^H x_leaf.
template <bool ACC>
__global__ void __launch_bounds__(MV_THREADS) mv_phase1(const WorkItem* items,
                                                       const DevChunk* hdr,
                                                       const float2* __restrict__ arena,
                                                       const typename MvT<ACC>::C2* __restrict__ xp,
                                                       typename MvT<ACC>::C2* t) {
    using R = typename MvT<ACC>::R;
    using C4 = typename MvT<ACC>::C4;
    const WorkItem it = items[blockIdx.x];
    __shared__ DevChunk sh_hdr[MAX_ITEM_CHUNKS];
    for (int i = threadIdx.x; i < it.last - it.first; i += MV_THREADS) sh_hdr[i] = hdr[it.first + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // this lane's x values (row pairs lane, lane+32, lane+64)
    C4 xv[PAIRS_PER_LANE];
#pragma unroll
    for (int q = 0; q < PAIRS_PER_LANE; ++q) {
        const int r = 2 * (lane + 32 * q);
        C4 v = {0, 0, 0, 0};
        if (r < it.rows) {
            v.x = xp[it.dof + r].x;
            v.y = xp[it.dof + r].y;
            if (r + 1 < it.rows) {
                v.z = xp[it.dof + r + 1].x;
                v.w = xp[it.dof + r + 1].y;
            }
        }
        xv[q] = v;
    }
    const int npair = (it.ld) >> 1;
    for (int ci = it.first; ci < it.last; ++ci) {
        const DevChunk ch = sh_hdr[ci - it.first];
        const float4* base = reinterpret_cast<const float4*>(arena + ch.data);
        for (int c = warp; c < ch.ncols; c += MV_WARPS) {
            const float4* col = base + (int64_t)c * (ch.ld >> 1);
            R re = 0, im = 0;
#pragma unroll
            for (int q = 0; q < PAIRS_PER_LANE; ++q) {
                const int pr = lane + 32 * q;
                if (pr < npair) {
                    const float4 v4 = ldg_stream(col + pr);
                    const R vx = v4.x, vy = v4.y, vz = v4.z, vw = v4.w;
                    // conj(v) * x
                    re = fma(vx, xv[q].x, fma(vy, xv[q].y, re));
                    im = fma(vx, xv[q].y, fma(-vy, xv[q].x, im));
                    re = fma(vz, xv[q].z, fma(vw, xv[q].w, re));
                    im = fma(vz, xv[q].w, fma(-vw, xv[q].z, im));
                }
            }
            re = red_sum(re);
            im = red_sum(im);
            if (lane == 0) atomic_add_c(t + ch.vec + c, re, im);
        }
    }
}

// Phase 2: y_leaf += sum over chunks of chunk * v, v = x (dense) or t (U).
template <bool ACC>
__global__ void __launch_bounds__(MV_THREADS) mv_phase2(const WorkItem* items,
                                                       const DevChunk* hdr,
                                                       const float2* __restrict__ arena,
                                                       const typename MvT<ACC>::C2* __restrict__ xp,
                                                       const typename MvT<ACC>::C2* __restrict__ t,
                                                       typename MvT<ACC>::C2* yp) {
    using R = typename MvT<ACC>::R;
    using C2 = typename MvT<ACC>::C2;
    using C4 = typename MvT<ACC>::C4;
    __shared__ C4 part[MV_WARPS][MAX_LD / 2];
    const WorkItem it = items[blockIdx.x];
    __shared__ DevChunk sh_hdr[MAX_ITEM_CHUNKS];
    for (int i = threadIdx.x; i < it.last - it.first; i += MV_THREADS) sh_hdr[i] = hdr[it.first + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int npair = it.ld >> 1;
    C4 acc[PAIRS_PER_LANE];
#pragma unroll
    for (int q = 0; q < PAIRS_PER_LANE; ++q) acc[q] = C4{0, 0, 0, 0};
    auto fma_col = [&](C4& s, const float4& a, const C2& v) {
        const R ax = a.x, ay = a.y, az = a.z, aw = a.w;
        s.x = fma(ax, v.x, fma(-ay, v.y, s.x));
        s.y = fma(ax, v.y, fma(ay, v.x, s.y));
        s.z = fma(az, v.x, fma(-aw, v.y, s.z));
        s.w = fma(az, v.y, fma(aw, v.x, s.w));
    };
    for (int ci = it.first; ci < it.last; ++ci) {
        const DevChunk ch = sh_hdr[ci - it.first];
        const float4* base = reinterpret_cast<const float4*>(arena + ch.data);
        const C2* v = (ch.kind == 0 ? xp : t) + ch.vec;
        int c = warp;
        // two columns per iteration for more loads in flight
        for (; c + MV_WARPS < ch.ncols; c += 2 * MV_WARPS) {
            const C2 v0 = v[c], v1 = v[c + MV_WARPS];
            const float4* col0 = base + (int64_t)c * (ch.ld >> 1);
            const float4* col1 = col0 + (int64_t)MV_WARPS * (ch.ld >> 1);
            float4 a0[PAIRS_PER_LANE], a1[PAIRS_PER_LANE];
#pragma unroll
            for (int q = 0; q < PAIRS_PER_LANE; ++q) {
                const int pr = lane + 32 * q;
                if (pr < npair) {
                    a0[q] = ldg_stream(col0 + pr);
                    a1[q] = ldg_stream(col1 + pr);
                }
            }
#pragma unroll
            for (int q = 0; q < PAIRS_PER_LANE; ++q) {
                const int pr = lane + 32 * q;
                if (pr < npair) {
                    fma_col(acc[q], a0[q], v0);
                    fma_col(acc[q], a1[q], v1);
                }
            }
        }
        for (; c < ch.ncols; c += MV_WARPS) {
            const C2 v0 = v[c];
            const float4* col0 = base + (int64_t)c * (ch.ld >> 1);
#pragma unroll
            for (int q = 0; q < PAIRS_PER_LANE; ++q) {
                const int pr = lane + 32 * q;
                if (pr < npair) fma_col(acc[q], ldg_stream(col0 + pr), v0);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PAIRS_PER_LANE; ++q) {
        const int pr = lane + 32 * q;
        if (pr < MAX_LD / 2) part[warp][pr] = acc[q];
    }
    __syncthreads();
    for (int pr = threadIdx.x; pr < npair; pr += MV_THREADS) {
        C4 s = part[0][pr];
        for (int w = 1; w < MV_WARPS; ++w) {
            s.x += part[w][pr].x;
            s.y += part[w][pr].y;
            s.z += part[w][pr].z;
            s.w += part[w][pr].w;
        }
        const int r = 2 * pr;
        if (r < it.rows) atomic_add_c(yp + it.dof + r, s.x, s.y);
        if (r + 1 < it.rows) atomic_add_c(yp + it.dof + r + 1, s.z, s.w);
    }
}

// ---- accurate product: FP32-stored entries, double-float sums ----
// x, t and the partial sums are carried as unevaluated pairs (hi, lo) of FP32
// numbers.  Each product a x_hi is split exactly into p + e with an FMA
// (e = a x_hi - p), p is added to the running hi part by an exact two-sum, and
// the rounding errors, e and a x_lo are gathered in the lo part (Dekker's
// product, Knuth's two-sum).  The sums carry about 44 significant bits,
// FP64-grade for the GMRES restart residuals, while the loops run on the FP32
// pipes (GB300's FP64 rate is 1/64 of its FP32 rate).  Every operation is an
// explicitly rounded intrinsic so the compiler cannot fuse the two-sums.
__device__ __forceinline__ void df_add_prod(float& h, float& l, float a, float xh, float xl) {
    const float p = __fmul_rn(a, xh);
    const float e = __fmaf_rn(a, xh, -p);
    const float t = __fadd_rn(h, p);
    const float bp = __fsub_rn(t, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    h = t;
    l = __fadd_rn(l, __fadd_rn(err, __fmaf_rn(a, xl, e)));
}
__device__ __forceinline__ void df_merge(float& h, float& l, float h2, float l2) {
    const float t = __fadd_rn(h, h2);
    const float bp = __fsub_rn(t, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(h2, bp));
    h = t;
    l = __fadd_rn(__fadd_rn(l, l2), err);
}
// Sums of four pairs over the warp, reduce-scatter style: after the exchange
// across lane bit 4 the lower half carries pairs 0, 1 and the upper half
// pairs 2, 3; after bit 3 each group of eight lanes carries one pair, and the
// last three exchanges complete it.  Lane group g = lane >> 3 ends with the
// total of pair g, in every lane of the group.
__device__ __forceinline__ void df_warp_sum4(float (&h)[4], float (&l)[4], int lane, float& oh,
                                             float& ol) {
    const bool up = lane & 16;
    float kh0 = up ? h[2] : h[0], kl0 = up ? l[2] : l[0];
    float kh1 = up ? h[3] : h[1], kl1 = up ? l[3] : l[1];
    const float sh0 = up ? h[0] : h[2], sl0 = up ? l[0] : l[2];
    const float sh1 = up ? h[1] : h[3], sl1 = up ? l[1] : l[3];
    df_merge(kh0, kl0, __shfl_xor_sync(0xffffffffu, sh0, 16), __shfl_xor_sync(0xffffffffu, sl0, 16));
    df_merge(kh1, kl1, __shfl_xor_sync(0xffffffffu, sh1, 16), __shfl_xor_sync(0xffffffffu, sl1, 16));
    const bool up8 = lane & 8;
    oh = up8 ? kh1 : kh0;
    ol = up8 ? kl1 : kl0;
    const float bh = up8 ? kh0 : kh1, bl = up8 ? kl0 : kl1;
    df_merge(oh, ol, __shfl_xor_sync(0xffffffffu, bh, 8), __shfl_xor_sync(0xffffffffu, bl, 8));
#pragma unroll
    for (int o = 4; o > 0; o >>= 1)
        df_merge(oh, ol, __shfl_xor_sync(0xffffffffu, oh, o), __shfl_xor_sync(0xffffffffu, ol, o));
}
// The same for two pairs: lane group lane >> 4 ends with the total of pair g.
__device__ __forceinline__ void df_warp_sum2(float h0, float l0, float h1, float l1, int lane,
                                             float& oh, float& ol) {
    const bool up = lane & 16;
    oh = up ? h1 : h0;
    ol = up ? l1 : l0;
    const float sh = up ? h0 : h1, sl = up ? l0 : l1;
    df_merge(oh, ol, __shfl_xor_sync(0xffffffffu, sh, 16), __shfl_xor_sync(0xffffffffu, sl, 16));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
        df_merge(oh, ol, __shfl_xor_sync(0xffffffffu, oh, o), __shfl_xor_sync(0xffffffffu, ol, o));
}
// complex128 -> (re_hi, im_hi, re_lo, im_lo)
__device__ __forceinline__ float4 df_split(double2 v) {
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
}

// t[vec + c] += V[:, c]^H x_leaf, double-float sums, FP64 atomics into t64.
__global__ void __launch_bounds__(MV_THREADS) mvdf_phase1(const WorkItem* items,
                                                         const DevChunk* hdr,
                                                         const float2* __restrict__ arena,
                                                         const float4* __restrict__ xdf,
                                                         double2* t64) {
    const WorkItem it = items[blockIdx.x];
    __shared__ DevChunk sh_hdr[MAX_ITEM_CHUNKS];
    for (int i = threadIdx.x; i < it.last - it.first; i += MV_THREADS) sh_hdr[i] = hdr[it.first + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 xa[PAIRS_PER_LANE], xb[PAIRS_PER_LANE];  // rows 2 pr and 2 pr + 1
#pragma unroll
    for (int q = 0; q < PAIRS_PER_LANE; ++q) {
        const int r = 2 * (lane + 32 * q);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        xa[q] = r < it.rows ? xdf[it.dof + r] : z;
        xb[q] = r + 1 < it.rows ? xdf[it.dof + r + 1] : z;
    }
    const int npair = it.ld >> 1;
    // conj(a) x for the lane's rows of one column, a = (a_re, a_im, b_re, b_im):
    // re += a_re x_re + a_im x_im, im += a_re x_im - a_im x_re (two rows per float4)
    auto col_dot = [&](const float4 (&v)[PAIRS_PER_LANE], float& rh, float& rl, float& ih, float& il) {
#pragma unroll
        for (int q = 0; q < PAIRS_PER_LANE; ++q) {
            if (lane + 32 * q < npair) {
                df_add_prod(rh, rl, v[q].x, xa[q].x, xa[q].z);
                df_add_prod(rh, rl, v[q].y, xa[q].y, xa[q].w);
                df_add_prod(ih, il, v[q].x, xa[q].y, xa[q].w);
                df_add_prod(ih, il, -v[q].y, xa[q].x, xa[q].z);
                df_add_prod(rh, rl, v[q].z, xb[q].x, xb[q].z);
                df_add_prod(rh, rl, v[q].w, xb[q].y, xb[q].w);
                df_add_prod(ih, il, v[q].z, xb[q].y, xb[q].w);
                df_add_prod(ih, il, -v[q].w, xb[q].x, xb[q].z);
            }
        }
    };
    auto load_col = [&](const float4* col, float4 (&v)[PAIRS_PER_LANE]) {
#pragma unroll
        for (int q = 0; q < PAIRS_PER_LANE; ++q)
            v[q] = (lane + 32 * q < npair) ? ldg_stream(col + lane + 32 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    // The totals go to t64 as two FP64 atomics per component (hi, then lo),
    // from lanes that each convert one FP32 part on the integer pipes.
    auto finish1 = [&](int64_t ti, float rh, float rl, float ih, float il) {
        float oh, ol;
        df_warp_sum2(rh, rl, ih, il, lane, oh, ol);
        if ((lane & 14) == 0) {
            double* dst = (lane & 16) ? &t64[ti].y : &t64[ti].x;
            atomicAdd(dst, f32_to_f64_bits((lane & 1) ? ol : oh));
        }
    };
    auto finish2 = [&](int64_t t0, int64_t t1, float (&h)[4], float (&l)[4]) {
        float oh, ol;
        df_warp_sum4(h, l, lane, oh, ol);
        if ((lane & 6) == 0) {
            double2* d = &t64[(lane & 16) ? t1 : t0];
            double* dst = (lane & 8) ? &d->y : &d->x;
            atomicAdd(dst, f32_to_f64_bits((lane & 1) ? ol : oh));
        }
    };
    for (int ci = it.first; ci < it.last; ++ci) {
        const DevChunk ch = sh_hdr[ci - it.first];
        const float4* base = reinterpret_cast<const float4*>(arena + ch.data);
        const int64_t cs = ch.ld >> 1;
        int c = warp;
        // two columns per pass: both columns' loads are in flight before the sums
        for (; c + MV_WARPS < ch.ncols; c += 2 * MV_WARPS) {
            float4 v0[PAIRS_PER_LANE], v1[PAIRS_PER_LANE];
            load_col(base + (int64_t)c * cs, v0);
            load_col(base + (int64_t)(c + MV_WARPS) * cs, v1);
            float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};  // re0, im0, re1, im1
            col_dot(v0, h[0], l[0], h[1], l[1]);
            col_dot(v1, h[2], l[2], h[3], l[3]);
            finish2(ch.vec + c, ch.vec + c + MV_WARPS, h, l);
        }
        for (; c < ch.ncols; c += MV_WARPS) {
            float4 v0[PAIRS_PER_LANE];
            load_col(base + (int64_t)c * cs, v0);
            float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
            col_dot(v0, rh, rl, ih, il);
            finish1(ch.vec + c, rh, rl, ih, il);
        }
    }
}

// y_leaf += sum over chunks of chunk * v (v = x or t as double-float), FP64 atomics into yp64.
__global__ void __launch_bounds__(MV_THREADS) mvdf_phase2(const WorkItem* items,
                                                         const DevChunk* hdr,
                                                         const float2* __restrict__ arena,
                                                         const float4* __restrict__ xdf,
                                                         const float4* __restrict__ tdf,
                                                         double2* yp64) {
    __shared__ float4 part[MV_WARPS][MAX_LD];  // (re_hi, re_lo, im_hi, im_lo) per row
    const WorkItem it = items[blockIdx.x];
    __shared__ DevChunk sh_hdr[MAX_ITEM_CHUNKS];
    for (int i = threadIdx.x; i < it.last - it.first; i += MV_THREADS) sh_hdr[i] = hdr[it.first + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int npair = it.ld >> 1;
    float4 sa[PAIRS_PER_LANE], sb[PAIRS_PER_LANE];  // rows 2 pr, 2 pr + 1: (re_h, re_l, im_h, im_l)
#pragma unroll
    for (int q = 0; q < PAIRS_PER_LANE; ++q) {
        sa[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        sb[q] = sa[q];
    }
    // rows += a w for the lane's rows of one column, a = (a_re, a_im, b_re, b_im):
    // re += a_re w_re - a_im w_im, im += a_re w_im + a_im w_re (two rows per float4)
    auto col_fma = [&](const float4 (&a)[PAIRS_PER_LANE], const float4& w) {
#pragma unroll
        for (int q = 0; q < PAIRS_PER_LANE; ++q) {
            if (lane + 32 * q < npair) {
                df_add_prod(sa[q].x, sa[q].y, a[q].x, w.x, w.z);
                df_add_prod(sa[q].x, sa[q].y, -a[q].y, w.y, w.w);
                df_add_prod(sa[q].z, sa[q].w, a[q].x, w.y, w.w);
                df_add_prod(sa[q].z, sa[q].w, a[q].y, w.x, w.z);
                df_add_prod(sb[q].x, sb[q].y, a[q].z, w.x, w.z);
                df_add_prod(sb[q].x, sb[q].y, -a[q].w, w.y, w.w);
                df_add_prod(sb[q].z, sb[q].w, a[q].z, w.y, w.w);
                df_add_prod(sb[q].z, sb[q].w, a[q].w, w.x, w.z);
            }
        }
    };
    auto load_col = [&](const float4* col, float4 (&a)[PAIRS_PER_LANE]) {
#pragma unroll
        for (int q = 0; q < PAIRS_PER_LANE; ++q)
            a[q] = (lane + 32 * q < npair) ? ldg_stream(col + lane + 32 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    for (int ci = it.first; ci < it.last; ++ci) {
        const DevChunk ch = sh_hdr[ci - it.first];
        const float4* base = reinterpret_cast<const float4*>(arena + ch.data);
        const float4* v = (ch.kind == 0 ? xdf : tdf) + ch.vec;  // (re_h, im_h, re_l, im_l)
        const int64_t cs = ch.ld >> 1;
        int c = warp;
        // two columns per pass: both columns' loads are in flight before the sums
        for (; c + MV_WARPS < ch.ncols; c += 2 * MV_WARPS) {
            const float4 w0 = __ldg(v + c), w1 = __ldg(v + c + MV_WARPS);
            float4 a0[PAIRS_PER_LANE], a1[PAIRS_PER_LANE];
            load_col(base + (int64_t)c * cs, a0);
            load_col(base + (int64_t)(c + MV_WARPS) * cs, a1);
            col_fma(a0, w0);
            col_fma(a1, w1);
        }
        for (; c < ch.ncols; c += MV_WARPS) {
            const float4 w0 = __ldg(v + c);
            float4 a0[PAIRS_PER_LANE];
            load_col(base + (int64_t)c * cs, a0);
            col_fma(a0, w0);
        }
    }
#pragma unroll
    for (int q = 0; q < PAIRS_PER_LANE; ++q) {
        const int r = 2 * (lane + 32 * q);
        if (r < MAX_LD) {
            part[warp][r] = sa[q];
            part[warp][r + 1] = sb[q];
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < it.rows; r += MV_THREADS) {
        float4 s = part[0][r];
        for (int w = 1; w < MV_WARPS; ++w) {
            const float4 u = part[w][r];
            df_merge(s.x, s.y, u.x, u.y);
            df_merge(s.z, s.w, u.z, u.w);
        }
        atomicAdd(&yp64[it.dof + r].x, (double)s.x + (double)s.y);
        atomicAdd(&yp64[it.dof + r].y, (double)s.z + (double)s.w);
    }
}

__global__ void gather_xdf_kernel(const int64_t* perm, const double2* x, float4* xdf, int64_t nc) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= 3 * nc) return;
    const int64_t p = q / 3, a = q - 3 * p;
    xdf[q] = df_split(x[3 * perm[p] + a]);
}

__global__ void split_df_kernel(const double2* t64, float4* tdf, int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) tdf[q] = df_split(t64[q]);
}

// ---- BF16 storage ----
__device__ __forceinline__ float2 bf2_to_f2(uint32_t u) {
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// ---- BF16 storage, streamed through shared memory ----
// Every work item is one contiguous byte range of the BF16 arena: the chunks of
// one leaf, all with the same leading dimension ld16, stored back to back, so
// the item is a column-major (ld16 x ncol) matrix.  One producer warp moves it
// into a ring of shared-memory stages with bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier per stage); eight consumer
// warps compute from the stages and release them through a second mbarrier
// per stage.  The bytes in flight per SM are set by the ring, not by the
// registers of the consumers.  Each wait gives up after PIPE_WAIT_NS, records
// an error code and lets the CTA finish; the producer always waits for its own
// copies before it exits.
//
// A consumer warp takes four columns of a stage at once, one per group of 8
// lanes; a lane covers the row quads sl, sl + 8, ... of its column (about 95 %
// of the lanes busy for the usual 150-row columns, where one column per warp
// leaves 40 % idle), so a stored entry costs one conversion and four FMAs and
// a column of phase 1 a three-step shuffle reduction.
// The number of stages in the ring (NS = 2, 3 or 4: 24-48 KB of the SM's
// shared memory per CTA) is a template parameter picked per GPU and workload
// by the autotuner (tune.cu); 3 without a tuning.
constexpr int S16_CONSUMERS = 4;
constexpr int S16_THREADS = 32 * (S16_CONSUMERS + 1);
constexpr int S16_COLS = 4 * S16_CONSUMERS;             // columns per stage: one per lane group
constexpr int S16_STAGE_BYTES = S16_COLS * MAX_LD * 4;  // 12 KB
constexpr int S16_QPL = MAX_LD / 4 / 8;                 // row quads per lane (48 quads / 8 lanes)
constexpr int MV_ERR_TIMEOUT = 1;

template <int NS>
struct S16Smem {
    static_assert(S16_CONSUMERS * MAX_LD * sizeof(float2) <= NS * S16_STAGE_BYTES,
                  "row sums fit in the stages");
    // the stages; once every stage is consumed, phase 2 reuses them for the
    // per-warp row sums (S16_CONSUMERS x MAX_LD float2)
    alignas(128) unsigned char stage[NS][S16_STAGE_BYTES];
    float2 w[MAX_ITEM_COLS];                   // phase 2: scale * v_j; phase 1: (t index bits, scale)
    DevChunk16 hdr[MAX_ITEM_CHUNKS];
    int32_t colstart[MAX_ITEM_CHUNKS + 1];
    int32_t ncol;
    alignas(8) uint64_t full[NS];
    uint64_t empty[NS];
};
// resident CTAs per SM the launch bounds ask for (48 KB stages allow three)
template <int NS> constexpr int s16_min_blocks() { return NS >= 4 ? 3 : 4; }

__device__ __forceinline__ void consumers_sync() { named_sync<1, 32 * S16_CONSUMERS>(); }

// PHASE 1: t[vec_j] += scale_j * V_j^H x_leaf;  PHASE 2: y_leaf += sum_j M_j scale_j v_j.
template <int PHASE, int NS>
__global__ void __launch_bounds__(S16_THREADS, s16_min_blocks<NS>()) mv16s_kernel(const WorkItem* items,
                                                           const DevChunk16* hdr,
                                                           const uint32_t* __restrict__ arena,
                                                           const float2* __restrict__ xp,
                                                           float2* t, float2* yp, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S16Smem<NS>& S = *reinterpret_cast<S16Smem<NS>*>(smem_raw);
    const WorkItem it = items[blockIdx.x];
    const int nch = it.last - it.first;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < nch; i += S16_THREADS) S.hdr[i] = hdr[it.first + i];
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], S16_CONSUMERS);
        }
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == 0) {  // column offsets of the chunks (exclusive scan, two chunks per lane)
        const int a0 = 2 * lane < nch ? S.hdr[2 * lane].ncols : 0;
        const int a1 = 2 * lane + 1 < nch ? S.hdr[2 * lane + 1].ncols : 0;
        int inc = a0 + a1;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const int exc = inc - a0 - a1;
        S.colstart[2 * lane] = exc;
        S.colstart[2 * lane + 1] = exc + a0;
        if (lane == 31) {
            S.colstart[MAX_ITEM_CHUNKS] = inc;
            S.ncol = inc;
        }
    }
    __syncthreads();
    const int ncol = S.ncol;
    const int ld16 = S.hdr[0].ld;
    const int colb = ld16 * 4;
    const int sc = S16_COLS;  // columns per stage
    const int nst = (ncol + sc - 1) / sc;
    if (warp == S16_CONSUMERS) {  // ---- producer ----
        if (lane == 0) {
            const unsigned char* src0 = reinterpret_cast<const unsigned char*>(arena + S.hdr[0].data);
            int issued = 0;
            for (int k = 0; k < nst; ++k) {
                const int s = k % NS;
                if (k >= NS && !mbar_wait(&S.empty[s], ((k / NS) - 1) & 1)) {
                    atomicExch(err, MV_ERR_TIMEOUT);
                    break;
                }
                const int g = min(sc, ncol - k * sc);
                const uint32_t bytes = (uint32_t)(g * colb);
                mbar_arrive_expect_tx(&S.full[s], bytes);
                bulk_g2s(S.stage[s], src0 + (size_t)k * sc * colb, bytes, &S.full[s]);
                ++issued;
            }
            for (int k = max(0, issued - NS); k < issued; ++k)  // own copies landed
                if (!mbar_wait(&S.full[k % NS], (k / NS) & 1)) atomicExch(err, MV_ERR_TIMEOUT);
        }
        return;
    }
    // ---- consumers: per-column table ----
    for (int ci = warp; ci < nch; ci += S16_CONSUMERS) {
        const DevChunk16 ch = S.hdr[ci];
        const int j0 = S.colstart[ci];
        for (int c = lane; c < ch.ncols; c += 32) {
            if (PHASE == 2) {
                const float2 v = __ldg((ch.kind == 0 ? xp : t) + ch.vec + c);
                S.w[j0 + c] = make_float2(v.x * ch.scale, v.y * ch.scale);
            } else {
                S.w[j0 + c] = make_float2(__int_as_float((int)(ch.vec + c)), ch.scale);
            }
        }
    }
    consumers_sync();
    const int nquad = (it.rows + 3) >> 2;
    const int nq8 = (nquad + 7) >> 3;  // quad rounds of the 8-lane groups (warp-uniform)
    const int ldq = ld16 >> 2;
    const int lg = lane >> 3, sl = lane & 7;
    // phase 1: x of this lane's rows; phase 2: the lane's partial row sums
    float2 xa[S16_QPL][4];
#pragma unroll
    for (int i = 0; i < S16_QPL; ++i)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = 4 * (sl + 8 * i) + e;
            xa[i][e] = (PHASE == 1 && r < it.rows) ? xp[it.dof + r] : make_float2(0.f, 0.f);
        }
    for (int k = 0; k < nst; ++k) {
        const int s = k % NS;
        if (!mbar_wait(&S.full[s], (k / NS) & 1)) {
            atomicExch(err, MV_ERR_TIMEOUT);
            break;
        }
        const int jb = k * sc;
        const int c = 4 * warp + lg;  // this lane group's column of the stage
        const bool valid = c < min(sc, ncol - jb);
        const uint4* col = reinterpret_cast<const uint4*>(S.stage[s]) + c * ldq;
        const float2 w = valid ? S.w[jb + c] : make_float2(0.f, 0.f);
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int i = 0; i < S16_QPL; ++i) {
            if (i < nq8) {
                const int qd = sl + 8 * i;
                const uint4 u = (valid && qd < nquad) ? col[qd] : make_uint4(0, 0, 0, 0);
                const uint32_t a4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 a = bf2_to_f2(a4[e]);
                    if (PHASE == 2) {  // rows += a w
                        float2& s2 = xa[i][e];
                        s2.x = fmaf(a.x, w.x, fmaf(-a.y, w.y, s2.x));
                        s2.y = fmaf(a.x, w.y, fmaf(a.y, w.x, s2.y));
                    } else {           // conj(a) x
                        const float2 xv = xa[i][e];
                        re = fmaf(a.x, xv.x, fmaf(a.y, xv.y, re));
                        im = fmaf(a.x, xv.y, fmaf(-a.y, xv.x, im));
                    }
                }
            }
        }
        if (PHASE == 1) {  // sum over the 8 lanes of the group
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, o);
                im += __shfl_xor_sync(0xffffffffu, im, o);
            }
            if (sl == 0 && valid) atomic_add_c(t + __float_as_int(w.x), re * w.y, im * w.y);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);
    }
    if (PHASE == 2) {
        // the four lane groups of a warp hold partial sums of the same rows
#pragma unroll
        for (int i = 0; i < S16_QPL; ++i)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float2& s2 = xa[i][e];
                s2.x += __shfl_xor_sync(0xffffffffu, s2.x, 8);
                s2.y += __shfl_xor_sync(0xffffffffu, s2.y, 8);
                s2.x += __shfl_xor_sync(0xffffffffu, s2.x, 16);
                s2.y += __shfl_xor_sync(0xffffffffu, s2.y, 16);
            }
        consumers_sync();  // every stage consumed: reuse them for the row sums
        float2(*part)[MAX_LD] = reinterpret_cast<float2(*)[MAX_LD]>(S.stage[0]);
        if (lg == 0) {
#pragma unroll
            for (int i = 0; i < S16_QPL; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) part[warp][4 * (sl + 8 * i) + e] = xa[i][e];
        }
        consumers_sync();
        for (int r = tid; r < it.rows; r += 32 * S16_CONSUMERS) {
            float2 s2 = part[0][r];
            for (int w = 1; w < S16_CONSUMERS; ++w) {
                s2.x += part[w][r].x;
                s2.y += part[w][r].y;
            }
            atomic_add_c(yp + it.dof + r, s2.x, s2.y);
        }
    }
}

__global__ void gather_hdr16_kernel(const DevChunk16* src, const int32_t* order, int64_t n,
                                    DevChunk16* dst) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) dst[q] = src[order[q]];
}

// FP32 chunk -> BF16 chunk.  Low-rank factors carry one scale per block and
// factor (the largest component magnitude of U, resp. V, over all chunks of
// the block); dense blocks are stored unscaled (BF16 keeps FP32's exponent
// range).  A V chunk also records its block's U scale (fold), so that a
// product may apply s_U s_V once to t = V^H x and use U's entries as stored.
struct ConvJob {
    int64_t src;    // FP32 arena offset
    int32_t ld32;
    int32_t chunk;  // index into chunks16
    int64_t slot;   // 2 block + (kind == V), -1 for dense
};
__device__ __forceinline__ float chunk_absmax(const ConvJob& J, const DevChunk16* ch,
                                              const float2* arena32, float* red) {
    const int rows = ch->rows, ncols = ch->ncols;
    const int64_t n = (int64_t)rows * ncols;
    float mx = 0.f;
    for (int64_t e = threadIdx.x; e < n; e += 256) {
        const int r = (int)(e % rows), c = (int)(e / rows);
        const float2 v = arena32[J.src + r + (int64_t)c * J.ld32];
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
    return mx;
}
__global__ void __launch_bounds__(256) block_absmax_kernel(const ConvJob* jobs, const float2* arena32,
                                                           const DevChunk16* chunks16, uint32_t* bmax) {
    __shared__ float red[8];
    const ConvJob J = jobs[blockIdx.x];
    if (J.slot < 0) return;
    const float mx = chunk_absmax(J, chunks16 + J.chunk, arena32, red);
    if (threadIdx.x == 0) atomicMax(bmax + J.slot, __float_as_uint(mx));  // non-negative floats order as integers
}
__global__ void __launch_bounds__(256) to_bf16_kernel(const ConvJob* jobs, const float2* arena32,
                                                      uint32_t* arena16, DevChunk16* chunks16,
                                                      const uint32_t* bmax) {
    const ConvJob J = jobs[blockIdx.x];
    DevChunk16* ch = chunks16 + J.chunk;
    const int rows = ch->rows, ncols = ch->ncols, ld16 = ch->ld;
    float scale = 1.f, fold = 1.f;
    if (J.slot >= 0) {
        const float m = __uint_as_float(bmax[J.slot]);
        scale = m > 0.f ? m : 1.f;
        if (J.slot & 1) {  // V chunk: the block's U scale
            const float mu = __uint_as_float(bmax[J.slot - 1]);
            fold = mu > 0.f ? mu : 1.f;
        }
    }
    const float inv = 1.f / scale;
    const int64_t n16 = (int64_t)ld16 * ncols;
    for (int64_t e = threadIdx.x; e < n16; e += 256) {
        const int r = (int)(e % ld16), c = (int)(e / ld16);
        uint32_t w = 0;
        if (r < rows) {
            const float2 v = arena32[J.src + r + (int64_t)c * J.ld32];
            const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(v.x * inv));
            const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(v.y * inv));
            w = lo | (hi << 16);
        }
        arena16[ch->data + e] = w;
    }
    if (threadIdx.x == 0) {
        ch->scale = scale;
        ch->fold = fold;
    }
}

__global__ void scatter_y64_kernel(const int64_t* perm, const double2* yp, double2* y, int64_t nc) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= 3 * nc) return;
    const int64_t p = q / 3, a = q - 3 * p;
    y[3 * perm[p] + a] = yp[q];
}

__global__ void gather_x_kernel(const int64_t* perm, const double2* x, float2* xp, int64_t nc) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= 3 * nc) return;
    const int64_t p = q / 3, a = q - 3 * p;
    const double2 v = x[3 * perm[p] + a];
    xp[q] = make_float2((float)v.x, (float)v.y);
}

__global__ void invert_perm_kernel(const int64_t* perm, int64_t nc, int64_t* iperm) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < nc) iperm[perm[p]] = p;
}

__global__ void scatter_y_kernel(const int64_t* perm, const float2* yp, double2* y, int64_t nc) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= 3 * nc) return;
    const int64_t p = q / 3, a = q - 3 * p;
    const float2 v = yp[q];
    y[3 * perm[p] + a] = make_double2(v.x, v.y);
}

struct StagedCopy {
    const float2* src;   // first row of the chunk's leaf in the staged block/factor
    int64_t src_ld;
    int64_t dst;
    int32_t ld, rows, ncols, pad_;
};

__global__ void __launch_bounds__(192) staged_copy_kernel(const StagedCopy* jobs, float2* arena) {
    const StagedCopy J = jobs[blockIdx.x];
    const int row = threadIdx.x;
    if (row >= J.ld) return;
    for (int c = 0; c < J.ncols; ++c)
        arena[J.dst + row + (int64_t)c * J.ld] =
            row < J.rows ? J.src[row + (int64_t)c * J.src_ld] : make_float2(0.f, 0.f);
}

// Splits each segment's chunk list into items of at most ~target bytes.
void make_items(const std::vector<int64_t>& begin, const std::vector<int32_t>& list,
                const std::vector<Chunk>& chunks, const MatvecPlan& plan, int64_t target,
                std::vector<WorkItem>& items, std::vector<int32_t>& order) {
    const int64_t nleaf = (int64_t)begin.size() - 1;
    for (int64_t l = 0; l < nleaf; ++l) {
        int64_t acc = 0;
        int32_t first = (int32_t)order.size();
        int64_t cols = 0;
        for (int64_t q = begin[l]; q < begin[l + 1]; ++q) {
            const Chunk& c = chunks[list[q]];
            if (c.ncols == 0) continue;
            if (c.ncols > MAX_ITEM_COLS) hm_throw(HM_ERR_UNSUPPORTED, "chunk wider than an item");
            if (cols + c.ncols > MAX_ITEM_COLS) {
                items.push_back({plan.leaf_dof_begin[l], plan.leaf_rows[l],
                                 (int32_t)hm_round_up(plan.leaf_rows[l], 2), first,
                                 (int32_t)order.size()});
                first = (int32_t)order.size();
                acc = 0;
                cols = 0;
            }
            order.push_back(list[q]);
            acc += (int64_t)c.ld * c.ncols * 8;
            cols += c.ncols;
            if (acc >= target || (int32_t)order.size() - first >= MAX_ITEM_CHUNKS) {
                items.push_back({plan.leaf_dof_begin[l], plan.leaf_rows[l],
                                 (int32_t)hm_round_up(plan.leaf_rows[l], 2), first,
                                 (int32_t)order.size()});
                first = (int32_t)order.size();
                acc = 0;
                cols = 0;
            }
        }
        if ((int32_t)order.size() > first)
            items.push_back({plan.leaf_dof_begin[l], plan.leaf_rows[l],
                             (int32_t)hm_round_up(plan.leaf_rows[l], 2), first,
                             (int32_t)order.size()});
    }
}

}  // namespace

MatvecPlan build_matvec_plan(const std::vector<hm_cluster>& cl, const std::vector<hm_block>& blk,
                             std::vector<int64_t>& t_off) {
    MatvecPlan P;
    // leaves in tree order
    std::vector<int64_t> leaves;
    for (int64_t c = 0; c < (int64_t)cl.size(); ++c)
        if (cl[c].is_leaf) leaves.push_back(c);
    std::sort(leaves.begin(), leaves.end(),
              [&](int64_t a, int64_t b) { return cl[a].begin < cl[b].begin; });
    // Storage segments: a leaf of up to MAX_LD / 3 points is one segment; a
    // larger leaf (N_leaf = 100 in Sec. 7) is cut into the fewest contiguous
    // point ranges of at most MAX_LD / 3 points, of nearly equal sizes.  Blocks
    // are cut along segments instead of leaves, so a chunk never has more than
    // MAX_LD rows (or, for dense chunks, columns); the tree and the partition
    // are unchanged.  Every cluster is a union of leaves, hence of segments.
    std::vector<int64_t> leaf_begin;
    const int64_t seg_max = MAX_LD / 3;
    for (int64_t c : leaves) {
        const int64_t np = cl[c].end - cl[c].begin;
        const int64_t k = std::max<int64_t>(1, hm_cdiv(np, seg_max));
        for (int64_t q = 0; q < k; ++q) {
            const int64_t b0 = cl[c].begin + q * np / k, b1 = cl[c].begin + (q + 1) * np / k;
            leaf_begin.push_back(b0);
            P.leaf_dof_begin.push_back(3 * b0);
            P.leaf_rows.push_back((int32_t)(3 * (b1 - b0)));
        }
    }
    const int64_t nleaf = (int64_t)leaf_begin.size();
    auto leaf_range = [&](int64_t c, int64_t& l0, int64_t& l1) {
        l0 = std::lower_bound(leaf_begin.begin(), leaf_begin.end(), cl[c].begin) - leaf_begin.begin();
        l1 = std::lower_bound(leaf_begin.begin(), leaf_begin.end(), cl[c].end) - leaf_begin.begin();
    };
    // t offsets, grouped by column cluster: the t entries of all blocks that
    // share sigma are one contiguous range, in block order
    t_off.assign(blk.size(), 0);
    std::vector<int64_t> by_sigma;
    for (size_t b = 0; b < blk.size(); ++b)
        if (blk[b].admissible) by_sigma.push_back((int64_t)b);
    std::stable_sort(by_sigma.begin(), by_sigma.end(),
                     [&](int64_t a, int64_t b) { return blk[a].sigma < blk[b].sigma; });
    int64_t toff = 0;
    for (int64_t b : by_sigma) {
        t_off[b] = toff;
        toff += blk[b].rank;
    }
    P.t_elems = toff;
    std::vector<std::vector<int32_t>> rows_of(nleaf), cols_of(nleaf);
    for (size_t b = 0; b < blk.size(); ++b) {
        const hm_cluster& t = cl[blk[b].tau];
        const hm_cluster& s = cl[blk[b].sigma];
        int64_t l0, l1, c0 = 0, c1 = 1;
        leaf_range(blk[b].tau, l0, l1);
        // dense blocks are cut along the column leaves too (chunks of at most
        // 3 x 64 columns: blocks stored dense after the ACA can be wide)
        if (!blk[b].admissible) leaf_range(blk[b].sigma, c0, c1);
        for (int64_t l = l0; l < l1; ++l) {
            for (int64_t lc = c0; lc < c1; ++lc) {
                Chunk c;
                c.rows = P.leaf_rows[l];
                c.ld = (int32_t)hm_round_up(c.rows, 2);
                c.block = (int64_t)b;
                c.sigma = blk[b].sigma;
                c.leaf_dof = P.leaf_dof_begin[l];
                if (!blk[b].admissible) {
                    c.kind = 0;
                    c.ncols = P.leaf_rows[lc];
                    c.vec = P.leaf_dof_begin[lc];
                } else {
                    c.kind = 1;
                    c.ncols = blk[b].rank;
                    c.vec = t_off[b];
                }
                c.data = -1;
                rows_of[l].push_back((int32_t)P.chunks.size());
                P.chunks.push_back(c);
            }
        }
        (void)t;
        (void)s;
        if (blk[b].admissible) {
            leaf_range(blk[b].sigma, l0, l1);
            for (int64_t l = l0; l < l1; ++l) {
                Chunk c;
                c.rows = P.leaf_rows[l];
                c.ld = (int32_t)hm_round_up(c.rows, 2);
                c.block = (int64_t)b;
                c.sigma = blk[b].sigma;
                c.leaf_dof = P.leaf_dof_begin[l];
                c.kind = 2;
                c.ncols = blk[b].rank;
                c.vec = t_off[b];
                c.data = -1;
                cols_of[l].push_back((int32_t)P.chunks.size());
                P.chunks.push_back(c);
            }
        }
    }
    // arena offsets: row-leaf streams first (dense chunks, then U), then V by column leaf
    int64_t off = 0;
    P.row_leaf_begin.push_back(0);
    for (int64_t l = 0; l < nleaf; ++l) {
        std::stable_sort(rows_of[l].begin(), rows_of[l].end(), [&](int32_t a, int32_t b) {
            return P.chunks[a].kind < P.chunks[b].kind;
        });
        for (int32_t id : rows_of[l]) {
            P.chunks[id].data = off;
            off += (int64_t)P.chunks[id].ld * P.chunks[id].ncols;
            P.row_items.push_back(id);
        }
        P.row_leaf_begin.push_back((int64_t)P.row_items.size());
    }
    // V chunks of a segment grouped by column cluster (block order inside a
    // group): the columns of the blocks that share sigma are one contiguous
    // run of every segment of sigma, in the same order, matching their t range
    P.col_leaf_begin.push_back(0);
    for (int64_t l = 0; l < nleaf; ++l) {
        std::stable_sort(cols_of[l].begin(), cols_of[l].end(), [&](int32_t a, int32_t b) {
            return P.chunks[a].sigma < P.chunks[b].sigma;
        });
        for (int32_t id : cols_of[l]) {
            P.chunks[id].data = off;
            off += (int64_t)P.chunks[id].ld * P.chunks[id].ncols;
            P.col_items.push_back(id);
        }
        P.col_leaf_begin.push_back((int64_t)P.col_items.size());
    }
    P.arena_elems = off;
    return P;
}

// Work items of the one-vector product (and of the accurate product): each
// segment's chunk list cut into items of about item_bytes (FP32 bytes),
// largest first; device copies of the items, their chunk order and the
// chunk headers in item order.  The buffers belong to the tiling and are
// replaced when it changes.
static void set_tiling(MatvecDev* m, const MatvecPlan& plan, int64_t item_bytes, cudaStream_t st) {
    std::vector<WorkItem> it1, it2;
    std::vector<int32_t> o1, o2;
    make_items(plan.col_leaf_begin, plan.col_items, plan.chunks, plan, item_bytes, it1, o1);
    make_items(plan.row_leaf_begin, plan.row_items, plan.chunks, plan, item_bytes, it2, o2);
    // largest items first (each item's bytes summed once, not per comparison)
    auto largest_first = [&](std::vector<WorkItem>& it, const std::vector<int32_t>& o) {
        std::vector<std::pair<int64_t, WorkItem>> kv;
        kv.reserve(it.size());
        for (const WorkItem& w : it) {
            int64_t s = 0;
            for (int32_t q = w.first; q < w.last; ++q)
                s += (int64_t)plan.chunks[o[q]].ld * plan.chunks[o[q]].ncols;
            kv.push_back({s, w});
        }
        std::stable_sort(kv.begin(), kv.end(),
                         [](const auto& a, const auto& b) { return a.first > b.first; });
        for (size_t i = 0; i < it.size(); ++i) it[i] = kv[i].second;
    };
    largest_first(it1, o1);
    largest_first(it2, o2);
    HM_CUDA(cudaStreamSynchronize(st));  // the old tiling is no longer in use
    for (DevBuf& d : m->tile_bufs) cudaFree(d.p);
    m->tile_bufs.clear();
    std::vector<DevBuf>& owner = m->tile_bufs;
    m->item_bytes = item_bytes;
    m->n1 = (int64_t)it1.size();
    m->n2 = (int64_t)it2.size();
    m->items1 = (WorkItem*)hm_dmalloc(owner, std::max<size_t>(it1.size(), 1) * sizeof(WorkItem), st, false);
    m->items2 = (WorkItem*)hm_dmalloc(owner, std::max<size_t>(it2.size(), 1) * sizeof(WorkItem), st, false);
    m->order1 = (int32_t*)hm_dmalloc(owner, std::max<size_t>(o1.size(), 1) * 4, st, false);
    m->order2 = (int32_t*)hm_dmalloc(owner, std::max<size_t>(o2.size(), 1) * 4, st, false);
    HM_CUDA(cudaMemcpyAsync(m->items1, it1.data(), it1.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(m->items2, it2.data(), it2.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(m->order1, o1.data(), o1.size() * 4, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(m->order2, o2.data(), o2.size() * 4, cudaMemcpyHostToDevice, st));
    std::vector<DevChunk> h1(o1.size()), h2(o2.size());
    for (size_t q = 0; q < o1.size(); ++q) h1[q] = m->dc[o1[q]];
    for (size_t q = 0; q < o2.size(); ++q) h2[q] = m->dc[o2[q]];
    m->hdr1 = (DevChunk*)hm_dmalloc(owner, std::max<size_t>(h1.size(), 1) * sizeof(DevChunk), st, false);
    m->hdr2 = (DevChunk*)hm_dmalloc(owner, std::max<size_t>(h2.size(), 1) * sizeof(DevChunk), st, false);
    HM_CUDA(cudaMemcpyAsync(m->hdr1, h1.data(), h1.size() * sizeof(DevChunk), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(m->hdr2, h2.data(), h2.size() * sizeof(DevChunk), cudaMemcpyHostToDevice, st));
    m->n_o1 = (int64_t)o1.size();
    m->n_o2 = (int64_t)o2.size();
    m->h_items1 = it1;
    m->h_items2 = it2;
    m->h_order1 = o1;
    m->h_order2 = o2;
    m->items1_full = m->items1;
    m->items2_full = m->items2;
    m->n1_full = m->n1;
    m->n2_full = m->n2;
    m->sel1 = m->sel2 = nullptr;
    HM_CUDA(cudaStreamSynchronize(st));  // host vectors h1, h2 leave scope
}

// Default work-item size: the largest power of two in [256 KB, 1 MB] of FP32
// bytes that still gives about ten waves of four resident CTAs per SM.  Each
// CTA pays a start (headers, the segment's x rows, its first copies) before
// its stream flows, so large operators run faster with fewer, larger items;
// small ones keep enough items to balance the SMs.  The BF16 layout follows
// this tiling, the FP32 products may retune it.
static int64_t default_item_bytes(int64_t arena_bytes) {
    int dev = 0, nsm = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t per = arena_bytes / (10LL * 4 * std::max(nsm, 1));
    int64_t ib = 256 * 1024;
    while (2 * ib <= per && ib < 1024 * 1024) ib *= 2;
    return ib;
}

MatvecDev* matvec_dev_create(const MatvecPlan& plan, int storage, std::vector<DevBuf>& owner,
                             cudaStream_t st) {
    MatvecDev* m = new MatvecDev();
    m->storage = storage;
    m->item_bytes = default_item_bytes(plan.arena_elems * (int64_t)sizeof(float2));
    m->arena_elems = plan.arena_elems;
    m->arena = (float2*)hm_dmalloc(owner, std::max<int64_t>(plan.arena_elems, 2) * sizeof(float2),
                                   st, true);
    std::vector<DevChunk> dc(plan.chunks.size());
    for (size_t i = 0; i < plan.chunks.size(); ++i) {
        const Chunk& c = plan.chunks[i];
        dc[i] = {c.data, c.vec, c.ld, c.ncols, c.kind, c.rows};
        if (c.kind == 0)
            m->dense_elems += (int64_t)c.ld * c.ncols;
        else
            m->lr_elems += (int64_t)c.ld * c.ncols;
        if (c.kind == 2)
            m->alg_v += (int64_t)c.rows * c.ncols;
        else
            m->alg_du += (int64_t)c.rows * c.ncols;
    }
    m->chunks = (DevChunk*)hm_dmalloc(owner, std::max<size_t>(dc.size(), 1) * sizeof(DevChunk), st,
                                      false);
    HM_CUDA(cudaMemcpyAsync(m->chunks, dc.data(), dc.size() * sizeof(DevChunk),
                            cudaMemcpyHostToDevice, st));
    m->dc = dc;
    set_tiling(m, plan, m->item_bytes, st);
    m->d_err = (int*)hm_dmalloc(owner, sizeof(int), st, true);
    m->t_elems = plan.t_elems;
    m->t = (float2*)hm_dmalloc(owner, std::max<int64_t>(plan.t_elems, 1) * sizeof(float2), st, true);
    m->t64 = (double2*)hm_dmalloc(owner, std::max<int64_t>(plan.t_elems, 1) * sizeof(double2), st, true);
    HM_CUDA(cudaStreamSynchronize(st));
    return m;
}

static void matvec_graph_reset(MatvecDev* m) {
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    if (m->graph) cudaGraphDestroy(m->graph);
    m->gexec = nullptr;
    m->graph = nullptr;
    m->g_gather = m->g_scatter = nullptr;
}

template <int NS>
static void s16_attributes() {
    HM_CUDA(cudaFuncSetAttribute(mv16s_kernel<1, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(S16Smem<NS>)));
    HM_CUDA(cudaFuncSetAttribute(mv16s_kernel<2, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(S16Smem<NS>)));
}

void matvec_make_bf16(MatvecDev* m, const MatvecPlan& plan, std::vector<DevBuf>& owner,
                      cudaStream_t st) {
    matvec_graph_reset(m);
    std::vector<DevChunk16> c16(plan.chunks.size());
    std::vector<ConvJob> jobs;
    int64_t off = 0;
    // Every work item starts on a multiple of its leading dimension, so that
    // the tensor-core product can address it as whole rows of a 2-D view of
    // the arena with row pitch ld16 (one TMA descriptor per ld16).
    std::vector<char> item_start(plan.chunks.size(), 0);
    for (const WorkItem& w : m->h_items1) item_start[m->h_order1[w.first]] = 1;
    for (const WorkItem& w : m->h_items2) item_start[m->h_order2[w.first]] = 1;
    // same order as the FP32 arena: row streams first, then V by column leaf
    std::vector<int32_t> seq(plan.row_items);
    seq.insert(seq.end(), plan.col_items.begin(), plan.col_items.end());
    for (int32_t id : seq) {
        const Chunk& c = plan.chunks[id];
        DevChunk16& d = c16[id];
        // >= 32 rows: a 64-element (128-byte) swizzle row never exceeds a column
        d.ld = (int32_t)std::max<int64_t>(hm_round_up(c.rows, 4), 32);
        if (item_start[id]) off = hm_round_up(off, d.ld);
        d.data = off;
        d.vec = c.vec;
        d.ncols = c.ncols;
        d.kind = c.kind;
        d.rows = c.rows;
        d.scale = 1.f;
        d.fold = 1.f;
        off += (int64_t)d.ld * c.ncols;
        if (c.ncols > 0) jobs.push_back({c.data, c.ld, id, c.kind == 0 ? -1 : 2 * c.block + (c.kind == 2)});
        if (c.ncols > 0) (c.kind == 2 ? m->nchunks_v : m->nchunks_du)++;
    }
    // the streamed kernels read every item as one contiguous column-major matrix
    auto check_items = [&](const std::vector<WorkItem>& items, const std::vector<int32_t>& order) {
        for (const WorkItem& w : items) {
            int64_t cols = 0;
            for (int32_t q = w.first; q < w.last; ++q) {
                const DevChunk16& a = c16[order[q]];
                cols += a.ncols;
                if (a.ld != c16[order[w.first]].ld || a.ld > MAX_LD || (a.data & 3))
                    hm_throw(HM_ERR_UNSUPPORTED, "BF16 item layout");
                if (q + 1 < w.last && c16[order[q + 1]].data != a.data + (int64_t)a.ld * a.ncols)
                    hm_throw(HM_ERR_UNSUPPORTED, "BF16 item not contiguous");
            }
            if (cols > MAX_ITEM_COLS || w.last - w.first > MAX_ITEM_CHUNKS)
                hm_throw(HM_ERR_UNSUPPORTED, "BF16 item too large");
            const DevChunk16& a = c16[order[w.first]];
            if (a.data % a.ld || a.data / a.ld > INT32_MAX - MAX_ITEM_COLS)
                hm_throw(HM_ERR_UNSUPPORTED, "BF16 item not on a row of its ld view");
        }
    };
    check_items(m->h_items1, m->h_order1);
    check_items(m->h_items2, m->h_order2);
    s16_attributes<2>();
    s16_attributes<3>();
    s16_attributes<4>();
    m->arena16_elems = off;
    m->nchunks = (int64_t)c16.size();
    // 256 bytes of slack: the block product's phase-2 view reads whole 128-byte
    // m-blocks, up to 126 bytes past the last stored column
    m->arena16 = (uint32_t*)hm_dmalloc(owner, std::max<int64_t>(off, 4) * 4 + 256, st, true);
    {  // TMA descriptors of the block product: [phase][ld16 / 4]
        std::vector<int32_t> lds;
        for (const WorkItem& w : m->h_items1) lds.push_back(c16[m->h_order1[w.first]].ld);
        for (const WorkItem& w : m->h_items2) lds.push_back(c16[m->h_order2[w.first]].ld);
        m->tmaps = hm_dmalloc(owner, TMAP_SETS * TMAP_PER_PHASE * 128, st, true);
        make_block_tmaps(m->tmaps, m->arena16, off, lds, st);
    }
    m->chunks16 = (DevChunk16*)hm_dmalloc(owner, std::max<size_t>(c16.size(), 1) * sizeof(DevChunk16),
                                          st, false);
    HM_CUDA(cudaMemcpyAsync(m->chunks16, c16.data(), c16.size() * sizeof(DevChunk16),
                            cudaMemcpyHostToDevice, st));
    if (!jobs.empty()) {
        ConvJob* d = nullptr;
        HM_CUDA(cudaMallocAsync((void**)&d, jobs.size() * sizeof(ConvJob), st));
        HM_CUDA(cudaMemcpyAsync(d, jobs.data(), jobs.size() * sizeof(ConvJob), cudaMemcpyHostToDevice, st));
        int64_t nblk = 0;
        for (const Chunk& c : plan.chunks) nblk = std::max<int64_t>(nblk, c.block + 1);
        uint32_t* bmax = nullptr;
        HM_CUDA(cudaMallocAsync((void**)&bmax, std::max<int64_t>(2 * nblk, 1) * 4, st));
        HM_CUDA(cudaMemsetAsync(bmax, 0, std::max<int64_t>(2 * nblk, 1) * 4, st));
        block_absmax_kernel<<<(unsigned)jobs.size(), 256, 0, st>>>(d, m->arena, m->chunks16, bmax);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
        to_bf16_kernel<<<(unsigned)jobs.size(), 256, 0, st>>>(d, m->arena, m->arena16, m->chunks16, bmax);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
        HM_CUDA(cudaFreeAsync(bmax, st));
        HM_CUDA(cudaFreeAsync(d, st));
    }
    m->hdr16_1 = (DevChunk16*)hm_dmalloc(owner, std::max<int64_t>(m->n_o1, 1) * sizeof(DevChunk16), st, false);
    m->hdr16_2 = (DevChunk16*)hm_dmalloc(owner, std::max<int64_t>(m->n_o2, 1) * sizeof(DevChunk16), st, false);
    if (m->n_o1) {
        gather_hdr16_kernel<<<(unsigned)hm_cdiv(m->n_o1, 256), 256, 0, st>>>(m->chunks16, m->order1, m->n_o1, m->hdr16_1);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
    if (m->n_o2) {
        gather_hdr16_kernel<<<(unsigned)hm_cdiv(m->n_o2, 256), 256, 0, st>>>(m->chunks16, m->order2, m->n_o2, m->hdr16_2);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
    make_block_items(m, plan, c16, owner, st);
    HM_CUDA(cudaStreamSynchronize(st));
    m->storage = HM_STORE_BF16;
}

void matvec_dev_destroy(MatvecDev* m) {
    if (!m) return;
    matvec_graph_reset(m);
    for (DevBuf& d : m->tile_bufs) cudaFree(d.p);
    if (m->xb) cudaFree(m->xb);
    if (m->ym) cudaFree(m->ym);
    if (m->iperm) cudaFree(m->iperm);
    if (m->tm) cudaFree(m->tm);
    if (m->t16) cudaFree(m->t16);
    if (m->tmap_xb) cudaFree(m->tmap_xb);
    delete m;
}
void* matvec_arena(MatvecDev* m) { return m->arena; }
int64_t matvec_stored_bytes(const MatvecDev* m) {
    return m->arena16 ? m->arena16_elems * 4 : m->arena_elems * 8;
}
int64_t matvec_dense_bytes(const MatvecDev* m) { return m->dense_elems * 8; }

template <int PHASE, int NS>
static void launch_s16(MatvecDev* m, const float2* xp, float2* yp, cudaStream_t st) {
    const int64_t n = PHASE == 1 ? m->n1 : m->n2;
    mv16s_kernel<PHASE, NS><<<(unsigned)n, S16_THREADS, sizeof(S16Smem<NS>), st>>>(
        PHASE == 1 ? m->items1 : m->items2, PHASE == 1 ? m->hdr16_1 : m->hdr16_2, m->arena16, xp,
        m->t, yp, m->d_err);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
}

template <int PHASE>
static void launch_s16_ns(MatvecDev* m, const float2* xp, float2* yp, cudaStream_t st) {
    switch (m->s16_nstage) {
        case 2: return launch_s16<PHASE, 2>(m, xp, yp, st);
        case 4: return launch_s16<PHASE, 4>(m, xp, yp, st);
        default: return launch_s16<PHASE, 3>(m, xp, yp, st);
    }
}

void matvec_phase1(MatvecDev* m, const float2* xp, cudaStream_t st) {
    if (m->t_elems) HM_CUDA(cudaMemsetAsync(m->t, 0, m->t_elems * sizeof(float2), st));
    if (m->n1 && m->arena16) {
        launch_s16_ns<1>(m, xp, nullptr, st);
    } else if (m->n1) {
        mv_phase1<false><<<(unsigned)m->n1, MV_THREADS, 0, st>>>(m->items1, m->hdr1,
                                                                m->arena, xp, m->t);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
}

void matvec_phase2(MatvecDev* m, const float2* xp, float2* yp, int64_t ndof, cudaStream_t st) {
    HM_CUDA(cudaMemsetAsync(yp, 0, ndof * sizeof(float2), st));
    if (m->n2 && m->arena16) {
        launch_s16_ns<2>(m, xp, yp, st);
    } else if (m->n2) {
        mv_phase2<false><<<(unsigned)m->n2, MV_THREADS, 0, st>>>(m->items2, m->hdr2,
                                                                m->arena, xp, m->t, yp);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
}

void matvec_tree_order(MatvecDev* m, const float2* xp, float2* yp, int64_t ndof, cudaStream_t st) {
    matvec_phase1(m, xp, st);
    matvec_phase2(m, xp, yp, ndof, st);
}

void matvec_accurate(MatvecDev* m, const int64_t* d_perm, const double2* x, double2* xp64,
                     double2* yp64, double2* y, int64_t nc, cudaStream_t st) {
    const int64_t n = 3 * nc;
    const unsigned nb = (unsigned)hm_cdiv(n, 256);
    // xp64 (3 nc complex128 = 16 B each) holds x in tree order as double-float pairs
    float4* xdf = reinterpret_cast<float4*>(xp64);
    gather_xdf_kernel<<<nb, 256, 0, st>>>(d_perm, x, xdf, nc);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    if (m->t_elems) HM_CUDA(cudaMemsetAsync(m->t64, 0, m->t_elems * sizeof(double2), st));
    HM_CUDA(cudaMemsetAsync(yp64, 0, n * sizeof(double2), st));
    if (m->n1) {
        mvdf_phase1<<<(unsigned)m->n1, MV_THREADS, 0, st>>>(m->items1, m->hdr1, m->arena, xdf,
                                                            m->t64);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
    if (m->t_elems) {  // t as double-float pairs, in place (16 B either way)
        split_df_kernel<<<(unsigned)hm_cdiv(m->t_elems, 256), 256, 0, st>>>(
            m->t64, reinterpret_cast<float4*>(m->t64), m->t_elems);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
    if (m->n2) {
        mvdf_phase2<<<(unsigned)m->n2, MV_THREADS, 0, st>>>(m->items2, m->hdr2, m->arena, xdf,
                                                            reinterpret_cast<const float4*>(m->t64),
                                                            yp64);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
    scatter_y64_kernel<<<nb, 256, 0, st>>>(d_perm, yp64, y, nc);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
}

void matvec_alg_bytes(const MatvecDev* m, int64_t ndof, int64_t out[3]) {
    const int64_t v = 8;  // complex64 vectors (x, t, y in tree order)
    if (m->arena16) {     // 4 bytes per stored entry + one FP32 scale per chunk
        out[0] = 4 * m->alg_v + 4 * m->nchunks_v + v * (ndof + m->t_elems);
        out[1] = 4 * m->alg_du + 4 * m->nchunks_du + v * (ndof + m->t_elems + ndof);
        out[2] = 4 * (m->alg_v + m->alg_du) + 4 * (m->nchunks_v + m->nchunks_du) + 2 * 16 * ndof;
        return;
    }
    out[0] = v * (m->alg_v + ndof + m->t_elems);
    out[1] = v * (m->alg_du + ndof + m->t_elems + ndof);
    out[2] = v * (m->alg_v + m->alg_du) + 2 * 16 * ndof;  // complex128 x in, y out
}

void matvec_ensure_iperm(MatvecDev* m, const int64_t* d_perm, int64_t nc, cudaStream_t st) {
    if (m->iperm) return;
    HM_CUDA(cudaMalloc((void**)&m->iperm, (size_t)std::max<int64_t>(nc, 1) * 8));
    invert_perm_kernel<<<(unsigned)hm_cdiv(nc, 256), 256, 0, st>>>(d_perm, nc, m->iperm);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
}

void launch_gather_x(const int64_t* d_perm, const double2* x, float2* xp, int64_t nc,
                     cudaStream_t st) {
    gather_x_kernel<<<(unsigned)hm_cdiv(3 * nc, 256), 256, 0, st>>>(d_perm, x, xp, nc);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
}

void launch_scatter_y(const int64_t* d_perm, const float2* yp, double2* y, int64_t nc,
                      cudaStream_t st) {
    scatter_y_kernel<<<(unsigned)hm_cdiv(3 * nc, 256), 256, 0, st>>>(d_perm, yp, y, nc);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
}

void copy_staged_chunks(MatvecDev* m, const MatvecPlan& plan, const std::vector<hm_block>& blk,
                        const std::vector<hm_cluster>& cl, const std::vector<const float2*>& src_u,
                        const std::vector<const float2*>& src_v, cudaStream_t st) {
    std::vector<StagedCopy> jobs;
    for (const Chunk& c : plan.chunks) {
        if (c.ncols == 0) continue;
        const hm_block& b = blk[c.block];
        const hm_cluster& t = cl[b.tau];
        const hm_cluster& s = cl[b.sigma];
        const float2* base = c.kind == 2 ? src_v[c.block] : src_u[c.block];
        if (!base) continue;
        const int64_t owner_begin = c.kind == 2 ? s.begin : t.begin;
        const int64_t owner_rows = 3 * (c.kind == 2 ? s.end - s.begin : t.end - t.begin);
        const int64_t col0 = c.kind == 0 ? c.vec - 3 * s.begin : 0;  // dense: the chunk's first column
        StagedCopy J;
        J.src = base + (c.leaf_dof - 3 * owner_begin) + col0 * owner_rows;
        J.src_ld = owner_rows;
        J.dst = c.data;
        J.ld = c.ld;
        J.rows = c.rows;
        J.ncols = c.ncols;
        J.pad_ = 0;
        if (J.ld > MAX_LD) hm_throw(HM_ERR_UNSUPPORTED, "chunk above MAX_LD rows");
        jobs.push_back(J);
    }
    if (jobs.empty()) return;
    StagedCopy* d = nullptr;
    HM_CUDA(cudaMallocAsync((void**)&d, jobs.size() * sizeof(StagedCopy), st));
    HM_CUDA(cudaMemcpyAsync(d, jobs.data(), jobs.size() * sizeof(StagedCopy), cudaMemcpyHostToDevice, st));
    staged_copy_kernel<<<(unsigned)jobs.size(), 192, 0, st>>>(d, m->arena);
    HM_CUDA(cudaGetLastError());
    HM_LAUNCHED();
    HM_CUDA(cudaFreeAsync(d, st));
}

// The product through its CUDA graph.  The graph is captured on a private
// stream (capture is not allowed on the legacy default stream) and launched on
// st; a call with other x / y pointers rewrites only the gather and scatter
// kernel nodes.
// Captures gather, both phases and scatter as the handle's product graph
// (x and y may be null: the first product re-points those two nodes).
static void graph_capture(MatvecDev* m, const int64_t* d_perm, const double2* x, float2* xp,
                          float2* yp, double2* y, int64_t nc) {
    {
        cudaStream_t cs = nullptr;
        HM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const long long before = g_hm_launches.load();
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            HM_CUDA(e);
        }
        try {
            launch_gather_x(d_perm, x, xp, nc, cs);
            matvec_tree_order(m, xp, yp, 3 * nc, cs);
            launch_scatter_y(d_perm, yp, y, nc, cs);
        } catch (...) {
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            g_hm_launches.store(before);
            throw;
        }
        e = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        HM_CUDA(e);
        m->g_kernels = g_hm_launches.load() - before;
        g_hm_launches.store(before);
        m->graph = g;
        size_t nn = 0;
        HM_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        HM_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            HM_CUDA(cudaGraphNodeGetType(nd, &ty));
            if (ty != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams p;
            HM_CUDA(cudaGraphKernelNodeGetParams(nd, &p));
            if (p.func == (void*)gather_x_kernel) m->g_gather = nd;
            if (p.func == (void*)scatter_y_kernel) m->g_scatter = nd;
        }
        if (!m->g_gather || !m->g_scatter) {
            matvec_graph_reset(m);
            hm_throw(HM_ERR_CUDA, "matvec graph: gather/scatter nodes not found");
        }
        e = cudaGraphInstantiate(&m->gexec, g, 0);
        if (e != cudaSuccess) {
            matvec_graph_reset(m);
            HM_CUDA(e);
        }
        m->g_x = x;
        m->g_y = y;
    }
}

void matvec_graph_prepare(MatvecDev* m, const int64_t* d_perm, float2* xp, float2* yp, int64_t nc) {
    if (!m->gexec) graph_capture(m, d_perm, nullptr, xp, yp, nullptr, nc);
}

void matvec_graph(MatvecDev* m, const int64_t* d_perm, const double2* x, float2* xp, float2* yp,
                  double2* y, int64_t nc, cudaStream_t st) {
    const unsigned nb = (unsigned)hm_cdiv(3 * nc, 256);
    if (!m->gexec) {
        graph_capture(m, d_perm, x, xp, yp, y, nc);
    } else {
        if (x != m->g_x) {
            const int64_t* a0 = d_perm;
            const double2* a1 = x;
            float2* a2 = xp;
            int64_t a3 = nc;
            void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&a3};
            cudaKernelNodeParams p = {};
            p.func = (void*)gather_x_kernel;
            p.gridDim = dim3(nb);
            p.blockDim = dim3(256);
            p.sharedMemBytes = 0;
            p.kernelParams = args;
            p.extra = nullptr;
            HM_CUDA(cudaGraphExecKernelNodeSetParams(m->gexec, m->g_gather, &p));
            m->g_x = x;
        }
        if (y != m->g_y) {
            const int64_t* a0 = d_perm;
            const float2* a1 = yp;
            double2* a2 = y;
            int64_t a3 = nc;
            void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&a3};
            cudaKernelNodeParams p = {};
            p.func = (void*)scatter_y_kernel;
            p.gridDim = dim3(nb);
            p.blockDim = dim3(256);
            p.sharedMemBytes = 0;
            p.kernelParams = args;
            p.extra = nullptr;
            HM_CUDA(cudaGraphExecKernelNodeSetParams(m->gexec, m->g_scatter, &p));
            m->g_y = y;
        }
    }
    HM_CUDA(cudaGraphLaunch(m->gexec, st));
    g_hm_launches.fetch_add(m->g_kernels, std::memory_order_relaxed);
}

// Error code of the streamed kernels since the last call (0 = none); resets it.
int matvec_take_error(MatvecDev* m, cudaStream_t st) {
    PinnedInt flag;
    matvec_queue_error(m, flag.p, st);
    HM_CUDA(cudaStreamSynchronize(st));
    return matvec_read_error(m, flag.p, st);
}

void matvec_queue_error(MatvecDev* m, int* pinned, cudaStream_t st) {
    HM_CUDA(cudaMemcpyAsync(pinned, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
}

int matvec_read_error(MatvecDev* m, const int* pinned, cudaStream_t st) {
    const int e = *pinned;
    if (e) HM_CUDA(cudaMemsetAsync(m->d_err, 0, sizeof(int), st));
    return e;
}

// Tunable launch parameters of the one-vector product (tune.cu): the stage
// count of the streamed BF16 kernels, and for FP32 storage the byte size of
// the work items (the BF16 arena is laid out along the build's items, so
// its tiling stays).  The product's CUDA graph is re-captured on next use.
void matvec_set_params(MatvecDev* m, const MatvecPlan& plan, int s16_nstage, int64_t item_bytes,
                       cudaStream_t st) {
    if (s16_nstage < 2 || s16_nstage > 4) hm_throw(HM_ERR_ARG, "stage count must be 2, 3 or 4");
    if (item_bytes < 16 * 1024 || item_bytes > 16 * 1024 * 1024)
        hm_throw(HM_ERR_ARG, "item bytes out of range");
    HM_CUDA(cudaStreamSynchronize(st));
    matvec_graph_reset(m);
    m->s16_nstage = s16_nstage;
    if (!m->arena16 && item_bytes != m->item_bytes) set_tiling(m, plan, item_bytes, st);
}

// Restricts the one-vector and accurate products to the work items whose
// rows (phase 2) or columns (phase 1) lie in an active segment of the vector
// (segment q = DOFs [dof_bounds[q], dof_bounds[q + 1]); blocks never straddle
// two segments of a joined batch).  Items of inactive segments are left out
// of the launches, so their parts of t and y stay zero.  All segments active
// restores the full item lists.  The product's graph is re-captured.
void matvec_select_segments(MatvecDev* m, const std::vector<int64_t>& dof_bounds,
                            const std::vector<int>& act, cudaStream_t st) {
    bool all = true;
    for (int a : act) all = all && a;
    HM_CUDA(cudaStreamSynchronize(st));
    matvec_graph_reset(m);
    if (all) {
        m->items1 = m->items1_full;
        m->items2 = m->items2_full;
        m->n1 = m->n1_full;
        m->n2 = m->n2_full;
        return;
    }
    if (!m->sel1) {
        m->sel1 = (WorkItem*)hm_dmalloc(m->tile_bufs, std::max<int64_t>(m->n1_full, 1) * sizeof(WorkItem), st, false);
        m->sel2 = (WorkItem*)hm_dmalloc(m->tile_bufs, std::max<int64_t>(m->n2_full, 1) * sizeof(WorkItem), st, false);
    }
    auto pick = [&](const std::vector<WorkItem>& all_items, WorkItem* dst, int64_t& n) {
        std::vector<WorkItem> keep;
        for (const WorkItem& w : all_items) {
            const int64_t q = std::upper_bound(dof_bounds.begin(), dof_bounds.end(), w.dof) - dof_bounds.begin() - 1;
            if (q >= 0 && q < (int64_t)act.size() && act[q]) keep.push_back(w);
        }
        n = (int64_t)keep.size();
        if (n) HM_CUDA(cudaMemcpyAsync(dst, keep.data(), n * sizeof(WorkItem), cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaStreamSynchronize(st));
    };
    pick(m->h_items1, m->sel1, m->n1);
    pick(m->h_items2, m->sel2, m->n2);
    m->items1 = m->sel1;
    m->items2 = m->sel2;
}

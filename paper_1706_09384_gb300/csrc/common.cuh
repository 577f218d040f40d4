// common.cuh — small device helpers shared by the hm CUDA sources:
// complex arithmetic on double2/float2, warp reductions, error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define HM_HD __host__ __device__ __forceinline__
#define HM_D __device__ __forceinline__

// ---- complex double (double2: x = re, y = im) ----
HM_HD double2 cz(double re, double im) { return make_double2(re, im); }
HM_HD double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
HM_HD double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
HM_HD double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
HM_HD double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
HM_HD double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
HM_HD double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// a * conj(b)
HM_HD double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conj(a) * b
HM_HD double2 cconjmul(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
HM_HD double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// acc += a * b
HM_HD void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc -= a * conj(b)
HM_HD void cfms_conj(double2& acc, double2 a, double2 b) {
    acc.x = fma(-a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
// acc += a * conj(b)
HM_HD void cfma_conjb(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
}
// acc -= conj(a) * b
HM_HD void cfms_conja(double2& acc, double2 a, double2 b) {
    acc.x = fma(-a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(-a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
HM_HD void cfma_conja(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}

// ---- complex float ----
HM_HD float2 cfmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
HM_HD void cffma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// acc += conj(a) * b
HM_HD void cffma_conja(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}

// ---- FP32 <-> FP64 on the integer pipes ----
// GB300 issues FP32/FP64 conversions on its narrow FP64 unit; moving the
// exponent and mantissa fields with integer operations leaves that unit free.
// FP32 -> FP64, exact like the conversion instruction; zero keeps its sign,
// subnormal, infinite and NaN inputs take the conversion.
HM_D double f32_to_f64_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint64_t sgn = (uint64_t)(b >> 31) << 63;
    if (e == 0u || e == 0xffu) return (b & 0x7fffffffu) ? (double)f : __longlong_as_double((long long)sgn);
    return __longlong_as_double(
        (long long)(sgn | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7fffffu) << 29)));
}
// FP64 -> FP32 rounded toward zero (the mantissa truncated to 23 bits) where
// the exponent lies in FP32's normal range; zero, values outside that range,
// infinities and NaN take the conversion (rounded to nearest).
HM_D float f64_to_f32_rz_bits(double d) {
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
    if (e < 897u || e > 1150u) return __double2float_rn(d);
    return __uint_as_float(((uint32_t)(b >> 63) << 31) | ((e - 896u) << 23) |
                           ((uint32_t)(b >> 29) & 0x7fffffu));
}

// ---- reductions ----
HM_D double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
HM_D float warp_sumf(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// argmax over (value, index): larger value wins, ties go to the lower index.
HM_D void argmax_merge(double& v, int64_t& i, double v2, int64_t i2) {
    if (v2 > v || (v2 == v && i2 >= 0 && (i < 0 || i2 < i))) {
        v = v2;
        i = i2;
    }
}
HM_D void warp_argmax(double& v, int64_t& i) {
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const long long i2 = __shfl_xor_sync(0xffffffffu, (long long)i, o);
        argmax_merge(v, i, v2, (int64_t)i2);
    }
}

static inline int64_t hm_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int64_t hm_round_up(int64_t a, int64_t b) { return hm_cdiv(a, b) * b; }

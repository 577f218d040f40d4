// green.cuh — device evaluation of the 3x3 elastodynamic Green's tensors.
//
// Eq. (elasto_U): U = (1/(rho w^2)) (curl curl_x[G_s I] - grad_x div_x[G_p I]),
// G_k = e^{i k r}/(4 pi r).  Off the source, curl curl = grad div - Lap and
// Lap G_k = -k^2 G_k give U = (1/mu)[G_s I + k_s^-2 grad grad (G_s - G_p)], i.e.
//   U_ab = psi(r) d_ab + chi(r) rh_a rh_b,   rh = (x - y)/r,
//   psi = (G_s + F'/(k_s^2 r))/mu,  chi = (F'' - F'/r)/(k_s^2 mu),  F = G_s - G_p.
// Eq. (elasto_T), component form of Sec. 5.3 (T_ab = C_agts d_{y_s} U_bt n_g,
// C = lam d_ag d_ts + mu (d_at d_gs + d_as d_gt)), with d_y = -d_x:
//   T = -mu (psi' + chi/r) [(rh.n) I + rh n^T] - 2 mu (chi' - 2 chi/r)(rh.n) rh rh^T
//       - [lam (psi' + chi' + 2 chi/r) + 2 mu chi/r] n rh^T.
// This is the a1..a5 structure printed in Sec. 2.3 with r-dependent coefficients.
#pragma once
#include "common.cuh"

struct GreenParams {
    double ks, kp;        // S and P wavenumbers (Sec. 1)
    double mu, lam;
    double inv_ks2;       // 1/k_s^2
    double diag;          // value of the i = j block (diag * I3)
    int kernel;           // 0 = U, 1 = T
    const double* w;      // device column weights in tree order (A = K W_y, Sec. 4), or null
    double ksr_switch;    // k_s r at and beyond which the tensor is evaluated in FP32
                          // (+inf: always FP64)
};

static inline GreenParams make_green_params(int kernel, double rho, double lam, double mu,
                                            double omega, double diag) {
    GreenParams p;
    p.ks = omega * sqrt(rho / mu);
    p.kp = omega * sqrt(rho / (lam + 2.0 * mu));
    p.mu = mu;
    p.lam = lam;
    p.inv_ks2 = 1.0 / (p.ks * p.ks);
    p.diag = diag;
    p.kernel = kernel;
    p.w = nullptr;
    p.ksr_switch = INFINITY;
    return p;
}

// d^n/dr^n of e^{ikr}/(4 pi r), n = 0..3, given ir = 1/r.
HM_D void helmholtz_derivs(double k, double r, double ir, double2 g[4]) {
    double s, c;
    sincos(k * r, &s, &c);
    const double a = ir * 0.079577471545947667884;  // 1/(4 pi r)
    const double2 e = make_double2(c * a, s * a);
    const double ir2 = ir * ir;
    g[0] = e;
    g[1] = cmul(e, make_double2(-ir, k));
    g[2] = cmul(e, make_double2(2.0 * ir2 - k * k, -2.0 * k * ir));
    g[3] = cmul(e, make_double2(3.0 * k * k * ir - 6.0 * ir2 * ir, 6.0 * k * ir2 - k * k * k));
}

// ---- FP32 evaluation away from the source ----
// The terms F'/(k_s^2 r) and F''/k_s^2 of psi and chi are each of size
// ~1/(k_s^2 r^3) and cancel to O(1/r): the relative rounding error of the sum
// grows like u / (k_s r)^2.  Where k_s r is at least ~1 that loss is gone:
// in FP32 (u = 6e-8) a U tensor is good to a few 1e-7 of its largest entry,
// a T tensor (whose coefficient psi' + chi/r cancels further) to 4e-6 at
// k_s r = 1 and below 1e-6 from k_s r = 2 (an FP32 emulation of these closed
// forms), all far below the eps_ACA the method uses; GB300 runs FP32 at 64
// times its FP64 rate.  The distance and the phase k r are formed in FP64 and
// the phase is reduced to [-pi, pi] there, so the FP32 sine and cosine see a
// small argument.
HM_D void helmholtz_derivs_f(double k, double r, float ir, float2 g[4]) {
    const double ph = k * r;
    const double red = fma(-6.283185307179586232, rint(ph * 0.15915494309189533577), ph);
    float s, c;
    sincosf((float)red, &s, &c);
    const float kf = (float)k;
    const float a = ir * 0.0795774715459476679f;  // 1/(4 pi r)
    const float2 e = make_float2(c * a, s * a);
    const float ir2 = ir * ir;
    g[0] = e;
    g[1] = cfmul(e, make_float2(-ir, kf));
    g[2] = cfmul(e, make_float2(2.0f * ir2 - kf * kf, -2.0f * kf * ir));
    g[3] = cfmul(e, make_float2(3.0f * kf * kf * ir - 6.0f * ir2 * ir,
                                6.0f * kf * ir2 - kf * kf * kf));
}

HM_D float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
HM_D float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
HM_D float2 f2scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
HM_D double2 f2d(float2 a) { return make_double2(f32_to_f64_bits(a.x), f32_to_f64_bits(a.y)); }

// The same closed forms as green_tensor below, in FP32 (r and the direction
// from FP64 differences of the coordinates).
HM_D void green_tensor_f32(const GreenParams& p, double r, const double rhd[3], const double* ny,
                           double2 G[9]) {
    const float ir = (float)(1.0 / r);
    const float rh[3] = {(float)rhd[0], (float)rhd[1], (float)rhd[2]};
    float2 gs[4], gp[4], F[4];
    helmholtz_derivs_f(p.ks, r, ir, gs);
    helmholtz_derivs_f(p.kp, r, ir, gp);
#pragma unroll
    for (int n = 0; n < 4; ++n) F[n] = f2sub(gs[n], gp[n]);
    const float imu = (float)(1.0 / p.mu), iks2 = (float)p.inv_ks2;
    const float2 psi = f2scale(f2add(gs[0], f2scale(F[1], ir * iks2)), imu);
    const float2 chi = f2scale(f2sub(F[2], f2scale(F[1], ir)), iks2 * imu);
    if (p.kernel == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                float2 v = f2scale(chi, rh[a] * rh[b]);
                if (a == b) v = f2add(v, psi);
                G[3 * a + b] = f2d(v);
            }
        return;
    }
    const float ir2 = ir * ir;
    const float mu = (float)p.mu, lam = (float)p.lam;
    const float2 dpsi =
        f2scale(f2add(gs[1], f2scale(f2sub(f2scale(F[2], ir), f2scale(F[1], ir2)), iks2)), imu);
    const float2 dchi = f2scale(f2add(f2sub(F[3], f2scale(F[2], ir)), f2scale(F[1], ir2)), iks2 * imu);
    const float nyf[3] = {(float)ny[0], (float)ny[1], (float)ny[2]};
    const float rn = rh[0] * nyf[0] + rh[1] * nyf[1] + rh[2] * nyf[2];
    const float2 chir = f2scale(chi, ir);
    const float2 c1 = f2scale(f2add(dpsi, chir), -mu);
    const float2 c2 = f2scale(f2sub(dchi, f2scale(chir, 2.0f)), -2.0f * mu);
    const float2 c3 = f2scale(f2add(f2scale(f2add(f2add(dpsi, dchi), f2scale(chir, 2.0f)), lam),
                                    f2scale(chir, 2.0f * mu)),
                              -1.0f);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float w1 = (a == b ? rn : 0.0f) + rh[a] * nyf[b];
            float2 v = f2scale(c1, w1);
            v = f2add(v, f2scale(c2, rn * rh[a] * rh[b]));
            v = f2add(v, f2scale(c3, nyf[a] * rh[b]));
            G[3 * a + b] = f2d(v);
        }
}

// G = K(x, y) (row-major 3x3); x != y required.  FP64, or FP32 where
// k_s r >= p.ksr_switch.
HM_D void green_tensor(const GreenParams& p, const double* x, const double* y, const double* ny,
                       double2 G[9]) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double ir = 1.0 / r;
    if (p.ks * r >= p.ksr_switch) {
        const double rhd[3] = {d0 * ir, d1 * ir, d2 * ir};
        green_tensor_f32(p, r, rhd, ny, G);
        return;
    }
    const double rh[3] = {d0 * ir, d1 * ir, d2 * ir};
    double2 gs[4], gp[4], F[4];
    helmholtz_derivs(p.ks, r, ir, gs);
    helmholtz_derivs(p.kp, r, ir, gp);
#pragma unroll
    for (int n = 0; n < 4; ++n) F[n] = csub(gs[n], gp[n]);
    const double imu = 1.0 / p.mu;
    const double2 psi = cscale(cadd(gs[0], cscale(F[1], ir * p.inv_ks2)), imu);
    const double2 chi = cscale(csub(F[2], cscale(F[1], ir)), p.inv_ks2 * imu);
    if (p.kernel == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                double2 v = cscale(chi, rh[a] * rh[b]);
                if (a == b) v = cadd(v, psi);
                G[3 * a + b] = v;
            }
        return;
    }
    const double ir2 = ir * ir;
    const double2 dpsi =
        cscale(cadd(gs[1], cscale(csub(cscale(F[2], ir), cscale(F[1], ir2)), p.inv_ks2)), imu);
    const double2 dchi =
        cscale(cadd(csub(F[3], cscale(F[2], ir)), cscale(F[1], ir2)), p.inv_ks2 * imu);
    const double rn = rh[0] * ny[0] + rh[1] * ny[1] + rh[2] * ny[2];
    const double2 chir = cscale(chi, ir);
    const double2 c1 = cscale(cadd(dpsi, chir), -p.mu);
    const double2 c2 = cscale(csub(dchi, cscale(chir, 2.0)), -2.0 * p.mu);
    const double2 c3 = cscale(cadd(cscale(cadd(cadd(dpsi, dchi), cscale(chir, 2.0)), p.lam),
                                   cscale(chir, 2.0 * p.mu)),
                              -1.0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const double w1 = (a == b ? rn : 0.0) + rh[a] * ny[b];
            double2 v = cscale(c1, w1);
            v = cadd(v, cscale(c2, rn * rh[a] * rh[b]));
            v = cadd(v, cscale(c3, ny[a] * rh[b]));
            G[3 * a + b] = v;
        }
}

// Column weight w_j (tree-order index j) applied to an off-diagonal block.
HM_D void apply_weight(const GreenParams& p, int64_t j, double2 G[9]) {
    if (!p.w) return;
    const double wj = p.w[j];
#pragma unroll
    for (int q = 0; q < 9; ++q) G[q] = cscale(G[q], wj);
}

// Block (i, j) of A: diag * I3 when the two points are the same index, else
// K(x_i, x_j) w_j.
HM_D void entry_block(const GreenParams& p, const double* pts, const double* nrm, int64_t i,
                      int64_t j, double2 G[9]) {
    if (i == j) {
#pragma unroll
        for (int q = 0; q < 9; ++q) G[q] = make_double2((q % 4 == 0) ? p.diag : 0.0, 0.0);
        return;
    }
    green_tensor(p, pts + 3 * i, pts + 3 * j, nrm ? nrm + 3 * j : nullptr, G);
    apply_weight(p, j, G);
}

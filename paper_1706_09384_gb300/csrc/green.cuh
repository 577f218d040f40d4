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

// G = K(x, y) (row-major 3x3); x != y required.
HM_D void green_tensor(const GreenParams& p, const double* x, const double* y, const double* ny,
                       double2 G[9]) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double ir = 1.0 / r;
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

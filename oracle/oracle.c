/*
 * oracle.c — plain FP64 CPU oracle for the H-matrix hot path of arXiv:1706.09384.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the bench).
 * The product path never links or calls it; it shares no code with the CUDA
 * path.  Everything here is written for readability, in the order and
 * notation of the paper; no blocking, fusion or reordering beyond what the
 * definitions state.  Compiled with -ffp-contract=off so that x86 and Arm
 * hosts round identically.
 *
 * Parity pins (tests/test_oracle_*.py) check every function below against
 * closed forms, invariants, library routines or brute force.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static inline cplx ld(const double* p) { return p[0] + I * p[1]; }
static inline void st(double* p, cplx z) { p[0] = creal(z); p[1] = cimag(z); }
static inline double abs2(cplx z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

/* ======================================================================
 * Green's tensors.
 *
 * Sec. 1 (Eq. elasto_U): U = (1/(rho w^2)) (curl curl_x[G_s I] - grad_x div_x[G_p I]),
 * G_k(r) = e^{i k r}/(4 pi r), k_p^2 = rho w^2/(lam + 2 mu), k_s^2 = rho w^2/mu.
 * With curl curl = grad div - Laplacian and (Laplacian + k^2) G_k = 0 off the
 * source, U = (1/mu) [G_s I + k_s^{-2} grad grad (G_s - G_p)].  For a radial
 * f(r), grad grad f = f'' rr + (f'/r)(I - rr) (r = x - y, rr = r^ r^^T), so
 *     U_ab = psi(r) delta_ab + chi(r) r^_a r^_b,
 *     psi = (1/mu) [G_s + F'/(k_s^2 r)],  chi = (1/mu) (F'' - F'/r)/k_s^2,
 * F = G_s - G_p.  This is the a1/a2 structure of Sec. 2.3 with r-dependent
 * coefficients.
 * ====================================================================== */

/* n-th r-derivative of G_k, n = 0..3. */
static void green_helmholtz_derivs(double k, double r, cplx g[4])
{
    const cplx e = cexp(I * k * r) / (4.0 * M_PI * r);
    const double ir = 1.0 / r;
    g[0] = e;
    g[1] = e * (I * k - ir);
    g[2] = e * (-k * k - 2.0 * I * k * ir + 2.0 * ir * ir);
    g[3] = e * (-I * k * k * k + 3.0 * k * k * ir + 6.0 * I * k * ir * ir - 6.0 * ir * ir * ir);
}

static void radial(double r, double rho, double lam, double mu, double omega,
                   cplx* psi, cplx* chi, cplx* dpsi, cplx* dchi)
{
    const double ks = omega * sqrt(rho / mu);             /* Sec. 1: k_s^2 = rho w^2 / mu */
    const double kp = omega * sqrt(rho / (lam + 2.0 * mu)); /* k_p^2 = rho w^2/(lam+2mu) */
    cplx gs[4], gp[4], F[4];
    green_helmholtz_derivs(ks, r, gs);
    green_helmholtz_derivs(kp, r, gp);
    for (int n = 0; n < 4; ++n) F[n] = gs[n] - gp[n];
    const double ks2 = ks * ks;
    *psi = (gs[0] + F[1] / (ks2 * r)) / mu;
    *chi = (F[2] - F[1] / r) / (ks2 * mu);
    *dpsi = (gs[1] + (F[2] / r - F[1] / (r * r)) / ks2) / mu;
    *dchi = (F[3] - F[2] / r + F[1] / (r * r)) / (ks2 * mu);
}

void or_radial(double r, double rho, double lam, double mu, double omega, double* out8)
{
    cplx a, b, c, d;
    radial(r, rho, lam, mu, omega, &a, &b, &c, &d);
    st(out8 + 0, a);
    st(out8 + 2, b);
    st(out8 + 4, c);
    st(out8 + 6, d);
}

/* K(x, y) for the configured kernel (entry block (i, j) of A in Eq. syst_a). */
static void green(const or_problem* pb, const double* x, const double* y, const double* ny,
                  cplx G[3][3])
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double rh[3] = {d[0] / r, d[1] / r, d[2] / r};
    cplx psi, chi, dpsi, dchi;
    radial(r, pb->rho, pb->lam, pb->mu, pb->omega, &psi, &chi, &dpsi, &dchi);
    if (pb->kernel == 0) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                G[a][b] = (a == b ? psi : 0.0) + chi * rh[a] * rh[b];
        return;
    }
    /* T_ab = C_{a g t s} d/dy_s U_{b t} n_g(y)  (Sec. 5.3 component form of
     * Eq. elasto_T), C = lam d_ag d_ts + mu (d_at d_gs + d_as d_gt).  With
     * d/dy = -d/dr along r^ and d(r^_b)/dx_s = (d_bs - r^_b r^_s)/r:
     *  T = -mu (psi' + chi/r) [(r^.n) I + r^ n^T]
     *      - 2 mu (chi' - 2 chi/r) (r^.n) r^ r^^T
     *      - [lam (psi' + chi' + 2 chi/r) + 2 mu chi/r] n r^^T. */
    const double mu = pb->mu, lam = pb->lam;
    const double rn = rh[0] * ny[0] + rh[1] * ny[1] + rh[2] * ny[2];
    const cplx c1 = -mu * (dpsi + chi / r);
    const cplx c2 = -2.0 * mu * (dchi - 2.0 * chi / r);
    const cplx c3 = -(lam * (dpsi + dchi + 2.0 * chi / r) + 2.0 * mu * chi / r);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            G[a][b] = c1 * ((a == b ? rn : 0.0) + rh[a] * ny[b]) + c2 * rn * rh[a] * rh[b] +
                      c3 * ny[a] * rh[b];
}

void or_green(const or_problem* pb, const double* x, const double* y, const double* ny,
              double* G18)
{
    cplx G[3][3];
    green(pb, x, y, ny, G);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) st(G18 + 2 * (3 * a + b), G[a][b]);
}

/* Block (i, j) of A: K(x_i, x_j) w_j off the diagonal (w_j = 1 without
 * weights; the column scaling W_y of the collocation matrix, Sec. 4),
 * diag_value * I3 on it.  The same cloud serves as x and y (Sec. 4). */
static void entry_block(const or_problem* pb, const double* pts, const double* nrm, int64_t i,
                        int64_t j, cplx G[3][3])
{
    if (i == j) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] = (a == b) ? pb->diag_value : 0.0;
        return;
    }
    green(pb, pts + 3 * i, pts + 3 * j, nrm ? nrm + 3 * j : NULL, G);
    if (pb->weights)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] *= pb->weights[j];
}

/* Block (i, j) between two clouds: K(x_i, y_j) w_j for a target point x_i of
 * X and a source point y_j of Y (normal and weight at y_j), diag_value * I3
 * where x_i and y_j coincide, so that X = Y reproduces entry_block. */
static void entry_block2(const or_problem* pb, const double* X, const double* Y, const double* nrmY,
                         int64_t i, int64_t j, cplx G[3][3])
{
    const double* x = X + 3 * i;
    const double* y = Y + 3 * j;
    if (x[0] == y[0] && x[1] == y[1] && x[2] == y[2]) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] = (a == b) ? pb->diag_value : 0.0;
        return;
    }
    green(pb, x, y, nrmY ? nrmY + 3 * j : NULL, G);
    if (pb->weights)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] *= pb->weights[j];
}

/* The 3 nx x 3 ny matrix between two clouds, row-major complex. */
void or_dense_matrix2(const or_problem* pb, const double* X, int64_t nx, const double* Y, int64_t ny,
                      const double* nrmY, double* A)
{
    const int64_t N = 3 * ny;
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j) {
            cplx G[3][3];
            entry_block2(pb, X, Y, nrmY, i, j, G);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) st(A + 2 * ((3 * i + a) * N + 3 * j + b), G[a][b]);
        }
}

void or_dense_matrix(const or_problem* pb, const double* pts, const double* nrm, int64_t nc,
                     double* A)
{
    const int64_t N = 3 * nc;
    for (int64_t i = 0; i < nc; ++i)
        for (int64_t j = 0; j < nc; ++j) {
            cplx G[3][3];
            entry_block(pb, pts, nrm, i, j, G);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) st(A + 2 * ((3 * i + a) * N + 3 * j + b), G[a][b]);
        }
}

void or_dense_rows_matvec(const or_problem* pb, const double* pts, const double* nrm,
                          int64_t nc, const int64_t* rows, int64_t nrows, const double* x,
                          double* out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t q = 0; q < nrows; ++q) {
        const int64_t i = rows[q] / 3;
        const int a = (int)(rows[q] % 3);
        cplx acc = 0.0;
        for (int64_t j = 0; j < nc; ++j) {
            cplx G[3][3];
            entry_block(pb, pts, nrm, i, j, G);
            for (int b = 0; b < 3; ++b) acc += G[a][b] * ld(x + 2 * (3 * j + b));
        }
        st(out + 2 * q, acc);
    }
}

/* ======================================================================
 * Cluster tree (Sec. 2.1, "Clustering of the unknowns"): the box enclosing
 * the points of a node is split in two along its largest dimension; the
 * subdivision stops once a node holds at most N_leaf points.
 * Readings where the paper is silent: the split is at the midpoint of the
 * tight box; ties between equal extents go to the lowest axis; a point goes
 * left iff its coordinate is < midpoint; children keep the parent order
 * (stable); left child first; a node whose box has zero extent, or whose
 * split would leave one side empty, stays a leaf.
 * ====================================================================== */
static void bbox(const double* pts, const int64_t* perm, int64_t b, int64_t e, double lo[3],
                 double hi[3])
{
    for (int a = 0; a < 3; ++a) {
        lo[a] = pts[3 * perm[b] + a];
        hi[a] = lo[a];
    }
    for (int64_t p = b + 1; p < e; ++p)
        for (int a = 0; a < 3; ++a) {
            const double v = pts[3 * perm[p] + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
}

static int64_t tree_rec(const double* pts, int64_t* perm, int64_t* tmp, int64_t leaf,
                        or_cluster* cl, int64_t* ncl, int64_t b, int64_t e, int level,
                        int64_t parent)
{
    const int64_t id = (*ncl)++;
    or_cluster* c = &cl[id];
    c->begin = b;
    c->end = e;
    c->level = level;
    c->parent = parent;
    c->child0 = c->child1 = -1;
    c->is_leaf = 1;
    bbox(pts, perm, b, e, c->lo, c->hi);
    if (e - b <= leaf) return id;
    int axis = 0;
    double ext = c->hi[0] - c->lo[0];
    for (int a = 1; a < 3; ++a)
        if (c->hi[a] - c->lo[a] > ext) {
            ext = c->hi[a] - c->lo[a];
            axis = a;
        }
    if (!(ext > 0.0)) return id;
    const double mid = (c->lo[axis] + c->hi[axis]) * 0.5;
    int64_t nl = 0, nr = 0;
    for (int64_t p = b; p < e; ++p)
        if (pts[3 * perm[p] + axis] < mid) nl++;
    if (nl == 0 || nl == e - b) return id;
    /* stable partition into tmp then back */
    int64_t il = 0;
    nr = 0;
    for (int64_t p = b; p < e; ++p) {
        if (pts[3 * perm[p] + axis] < mid)
            tmp[b + il++] = perm[p];
        else
            tmp[b + nl + nr++] = perm[p];
    }
    memcpy(perm + b, tmp + b, (size_t)(e - b) * sizeof(int64_t));
    c->is_leaf = 0;
    const int64_t c0 = tree_rec(pts, perm, tmp, leaf, cl, ncl, b, b + nl, level + 1, id);
    const int64_t c1 = tree_rec(pts, perm, tmp, leaf, cl, ncl, b + nl, e, level + 1, id);
    cl[id].child0 = c0;
    cl[id].child1 = c1;
    return id;
}

int64_t or_tree_build(const double* pts, int64_t nc, int64_t leaf, int64_t* perm, or_cluster* out)
{
    for (int64_t i = 0; i < nc; ++i) perm[i] = i;
    if (nc == 0) return 0;
    int64_t* tmp = (int64_t*)malloc((size_t)nc * sizeof(int64_t));
    int64_t ncl = 0;
    tree_rec(pts, perm, tmp, leaf < 1 ? 1 : leaf, out, &ncl, 0, nc, 0, -1);
    free(tmp);
    return ncl;
}

/* Sec. 6.1: diam_box(X) = (sum_a (max x_a - min x_a)^2)^{1/2}. */
double or_diam_box(const double* lo, const double* hi)
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a) s = s + (hi[a] - lo[a]) * (hi[a] - lo[a]);
    return sqrt(s);
}

/* Sec. 6.1: dist_box = distance between the closest faces of the boxes.  The
 * printed formula squares both differences unconditionally, which is not a
 * lower bound of dist for overlapping boxes; the reading used is the
 * positive part per axis: gap_a = max(0, lo1_a - hi2_a, lo2_a - hi1_a). */
double or_dist_box(const double* lo1, const double* hi1, const double* lo2, const double* hi2)
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double g = 0.0;
        if (lo1[a] - hi2[a] > g) g = lo1[a] - hi2[a];
        if (lo2[a] - hi1[a] > g) g = lo2[a] - hi1[a];
        s = s + g * g;
    }
    return sqrt(s);
}

/* Eq. admissibility_cond_bis: min(diam_box X, diam_box Y) < eta * dist_box(X, Y). */
int or_admissible_box(const double* lo1, const double* hi1, const double* lo2, const double* hi2,
                      double eta)
{
    const double d1 = or_diam_box(lo1, hi1), d2 = or_diam_box(lo2, hi2);
    const double dm = d1 < d2 ? d1 : d2;
    return dm < eta * or_dist_box(lo1, hi1, lo2, hi2);
}

/* Eq. admissibility_cond with the exact diameter and distance of the point sets. */
int or_admissible_exact(const double* X, int64_t nx, const double* Y, int64_t ny, double eta)
{
    double dx = 0.0, dy = 0.0, dist = INFINITY;
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < nx; ++j) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += (X[3 * i + a] - X[3 * j + a]) * (X[3 * i + a] - X[3 * j + a]);
            if (sqrt(s) > dx) dx = sqrt(s);
        }
    for (int64_t i = 0; i < ny; ++i)
        for (int64_t j = 0; j < ny; ++j) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += (Y[3 * i + a] - Y[3 * j + a]) * (Y[3 * i + a] - Y[3 * j + a]);
            if (sqrt(s) > dy) dy = sqrt(s);
        }
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += (X[3 * i + a] - Y[3 * j + a]) * (X[3 * i + a] - Y[3 * j + a]);
            if (sqrt(s) < dist) dist = sqrt(s);
        }
    return (dx < dy ? dx : dy) < eta * dist;
}

/* Sec. 2.1 "Subdivision of the matrix": starting from (root, root) each block
 * is subdivided until it is admissible or the leaf level is reached.  A pair
 * that is not admissible and has a leaf on either side is a dense leaf block
 * (Sec. 5.1: non-admissible blocks only at the leaf level, N_st <= N_leaf max).
 * Children are visited (t0,s0), (t0,s1), (t1,s0), (t1,s1). */
static void part_rec(const or_cluster* cl, double eta, int64_t t, int64_t s, or_block* out,
                     int64_t* nb)
{
    if (or_admissible_box(cl[t].lo, cl[t].hi, cl[s].lo, cl[s].hi, eta)) {
        if (out) {
            out[*nb].tau = t;
            out[*nb].sigma = s;
            out[*nb].admissible = 1;
            out[*nb].pad_ = 0;
        }
        (*nb)++;
        return;
    }
    if (cl[t].is_leaf || cl[s].is_leaf) {
        if (out) {
            out[*nb].tau = t;
            out[*nb].sigma = s;
            out[*nb].admissible = 0;
            out[*nb].pad_ = 0;
        }
        (*nb)++;
        return;
    }
    const int64_t tc[2] = {cl[t].child0, cl[t].child1};
    const int64_t sc[2] = {cl[s].child0, cl[s].child1};
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) part_rec(cl, eta, tc[u], sc[v], out, nb);
}

int64_t or_partition(const or_cluster* cl, int64_t ncl, double eta, or_block* out)
{
    if (ncl == 0) return 0;
    int64_t nb = 0;
    part_rec(cl, eta, 0, 0, out, &nb);
    return nb;
}

/* ======================================================================
 * Small dense linear algebra.
 * ====================================================================== */

/* One-sided Jacobi SVD (Hestenes) of a col-major M x N complex matrix,
 * M >= N: columns are orthogonalised pairwise by unitary plane rotations
 * until all pairs are orthogonal to working precision; singular values are
 * the column norms, sorted descending.  Uo (M x N) and Vo (N x N) optional. */
static int svd_jacobi(cplx* W, int64_t M, int64_t N, double* s, cplx* Vm)
{
    for (int64_t i = 0; i < N * N; ++i) Vm[i] = 0.0;
    for (int64_t i = 0; i < N; ++i) Vm[i + i * N] = 1.0;
    int converged = 0;
    for (int sweep = 0; sweep < 80 && !converged; ++sweep) {
        converged = 1;
        for (int64_t p = 0; p < N - 1; ++p)
            for (int64_t q = p + 1; q < N; ++q) {
                double alpha = 0.0, beta = 0.0;
                cplx gamma = 0.0;
                for (int64_t r = 0; r < M; ++r) {
                    alpha += abs2(W[r + p * M]);
                    beta += abs2(W[r + q * M]);
                    gamma += conj(W[r + p * M]) * W[r + q * M];
                }
                const double ag = cabs(gamma);
                if (ag == 0.0 || ag <= 1e-15 * sqrt(alpha * beta)) continue;
                converged = 0;
                const cplx ph = gamma / ag; /* e^{i phi} */
                const double zeta = (beta - alpha) / (2.0 * ag);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                /* [w_p, w_q] <- [w_p, w_q] J, J = [[c, sn], [-sn e^{-i phi}, c e^{-i phi}]] */
                const cplx phc = conj(ph);
                for (int64_t r = 0; r < M; ++r) {
                    const cplx wp = W[r + p * M], wq = W[r + q * M];
                    W[r + p * M] = c * wp - sn * phc * wq;
                    W[r + q * M] = sn * wp + c * phc * wq;
                }
                for (int64_t r = 0; r < N; ++r) {
                    const cplx vp = Vm[r + p * N], vq = Vm[r + q * N];
                    Vm[r + p * N] = c * vp - sn * phc * vq;
                    Vm[r + q * N] = sn * vp + c * phc * vq;
                }
            }
    }
    for (int64_t j = 0; j < N; ++j) {
        double nn = 0.0;
        for (int64_t r = 0; r < M; ++r) nn += abs2(W[r + j * M]);
        s[j] = sqrt(nn);
    }
    /* sort descending (selection sort keeps it obvious), permuting W and Vm */
    for (int64_t i = 0; i < N; ++i) {
        int64_t best = i;
        for (int64_t j = i + 1; j < N; ++j)
            if (s[j] > s[best]) best = j;
        if (best != i) {
            double ts = s[i];
            s[i] = s[best];
            s[best] = ts;
            for (int64_t r = 0; r < M; ++r) {
                cplx tw = W[r + i * M];
                W[r + i * M] = W[r + best * M];
                W[r + best * M] = tw;
            }
            for (int64_t r = 0; r < N; ++r) {
                cplx tv = Vm[r + i * N];
                Vm[r + i * N] = Vm[r + best * N];
                Vm[r + best * N] = tv;
            }
        }
    }
    return converged ? 0 : 1;
}

int or_svd_jacobi(const double* A, int64_t M, int64_t N, double* s, double* Uo, double* Vo)
{
    cplx* W = (cplx*)malloc((size_t)(M * N) * sizeof(cplx));
    cplx* Vm = (cplx*)malloc((size_t)(N * N) * sizeof(cplx));
    for (int64_t i = 0; i < M * N; ++i) W[i] = ld(A + 2 * i);
    const int rc = svd_jacobi(W, M, N, s, Vm);
    if (Uo)
        for (int64_t j = 0; j < N; ++j)
            for (int64_t r = 0; r < M; ++r)
                st(Uo + 2 * (r + j * M), s[j] > 0.0 ? W[r + j * M] / s[j] : 0.0);
    if (Vo)
        for (int64_t i = 0; i < N * N; ++i) st(Vo + 2 * i, Vm[i]);
    free(W);
    free(Vm);
    return rc;
}

/* Singular values of a 3x3 complex block (the sigma_1 >= sigma_2 >= sigma_3 of
 * Sec. 2.3, strategy 3) by the same one-sided Jacobi SVD. */
static void sv3(cplx B[3][3], double s[3])
{
    cplx W[9], Vm[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) W[a + 3 * b] = B[a][b];
    svd_jacobi(W, 3, 3, s, Vm);
}

void or_sv3(const double* M18, double* s3)
{
    cplx B[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) B[a][b] = ld(M18 + 2 * (3 * a + b));
    sv3(B, s3);
}

/* Householder QR of a col-major M x N complex matrix (M >= N): A = Q R with
 * Q (M x N) having orthonormal columns and R (N x N) upper triangular. */
static void qr_householder(const cplx* A, int64_t M, int64_t N, cplx* Q, cplx* R)
{
    cplx* W = (cplx*)malloc((size_t)(M * N) * sizeof(cplx));
    cplx* vs = (cplx*)calloc((size_t)(M * N), sizeof(cplx)); /* reflector j in column j */
    memcpy(W, A, (size_t)(M * N) * sizeof(cplx));
    for (int64_t j = 0; j < N; ++j) {
        double nx = 0.0;
        for (int64_t r = j; r < M; ++r) nx += abs2(W[r + j * M]);
        nx = sqrt(nx);
        cplx* v = vs + j * M;
        if (nx == 0.0) continue; /* H_j = I */
        const cplx x0 = W[j + j * M];
        const cplx ph = (cabs(x0) > 0.0) ? x0 / cabs(x0) : 1.0;
        const cplx alpha = -ph * nx; /* H x = alpha e1 */
        for (int64_t r = j; r < M; ++r) v[r] = W[r + j * M];
        v[j] -= alpha;
        double nv = 0.0;
        for (int64_t r = j; r < M; ++r) nv += abs2(v[r]);
        nv = sqrt(nv);
        for (int64_t r = j; r < M; ++r) v[r] /= nv;
        /* W[j:, j:] -= 2 v (v^H W[j:, j:]) */
        for (int64_t c = j; c < N; ++c) {
            cplx dot = 0.0;
            for (int64_t r = j; r < M; ++r) dot += conj(v[r]) * W[r + c * M];
            for (int64_t r = j; r < M; ++r) W[r + c * M] -= 2.0 * v[r] * dot;
        }
    }
    for (int64_t c = 0; c < N; ++c)
        for (int64_t r = 0; r < N; ++r) R[r + c * N] = (r <= c) ? W[r + c * M] : 0.0;
    /* Q = H_0 H_1 ... H_{N-1} [I_N; 0] */
    for (int64_t c = 0; c < N; ++c)
        for (int64_t r = 0; r < M; ++r) Q[r + c * M] = (r == c) ? 1.0 : 0.0;
    for (int64_t j = N - 1; j >= 0; --j) {
        const cplx* v = vs + j * M;
        for (int64_t c = 0; c < N; ++c) {
            cplx dot = 0.0;
            for (int64_t r = j; r < M; ++r) dot += conj(v[r]) * Q[r + c * M];
            for (int64_t r = j; r < M; ++r) Q[r + c * M] -= 2.0 * v[r] * dot;
        }
    }
    free(W);
    free(vs);
}

int or_qr_householder(const double* A, int64_t M, int64_t N, double* Q, double* R)
{
    cplx* a = (cplx*)calloc((size_t)(M * N) + 1, sizeof(cplx));
    cplx* q = (cplx*)malloc((size_t)(M * N) * sizeof(cplx));
    cplx* rr = (cplx*)malloc((size_t)(N * N) * sizeof(cplx));
    for (int64_t i = 0; i < M * N; ++i) a[i] = ld(A + 2 * i);
    qr_householder(a, M, N, q, rr);
    for (int64_t i = 0; i < M * N; ++i) st(Q + 2 * i, q[i]);
    for (int64_t i = 0; i < N * N; ++i) st(R + 2 * i, rr[i]);
    free(a);
    free(q);
    free(rr);
    return 0;
}

/* Inverse of a 3x3 complex block by the adjugate: gamma = R(i^, j^)^{-1}
 * (Sec. 2.2 step 2, block form of Sec. 2.3). */
static void inv3(cplx A[3][3], cplx B[3][3])
{
    const cplx c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    const cplx c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    const cplx c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const cplx det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    B[0][0] = c00 / det;
    B[1][0] = c01 / det;
    B[2][0] = c02 / det;
    B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
}

/* ======================================================================
 * Vector ACA (Sec. 2.2, partially pivoted ACA in six steps, with the
 * rank-3 update and sigma_3 pivot of Sec. 2.3, strategy 3).
 * A block source yields rows A(i,:) as 3 x 3n and columns A(:,j) as 3m x 3
 * (point indices local to the block).
 * ====================================================================== */
typedef struct {
    int kind; /* 0: explicit row-major matrix, 1: Green's kernel on points */
    int64_t m, n;
    const double* A; /* kind 0: 3m x 3n row-major complex */
    const or_problem* pb; /* kind 1 */
    const double* pts;
    const double* nrm;
    const int64_t* rows; /* global point index of local row point i */
    const int64_t* cols;
    const double* pts_y; /* kind 1, two clouds: source points (columns), else NULL */
    const double* nrm_y;
} block_src;

/* Block (i, j) of a kernel source: one cloud, or targets pts and sources pts_y. */
static void src_entry(const block_src* s, int64_t i, int64_t j, cplx G[3][3])
{
    if (s->pts_y)
        entry_block2(s->pb, s->pts, s->pts_y, s->nrm_y, s->rows[i], s->cols[j], G);
    else
        entry_block(s->pb, s->pts, s->nrm, s->rows[i], s->cols[j], G);
}

static void src_row(const block_src* s, int64_t i, cplx* R /* 3 x 3n row-major */)
{
    const int64_t n3 = 3 * s->n;
    if (s->kind == 0) {
        for (int a = 0; a < 3; ++a)
            for (int64_t c = 0; c < n3; ++c) R[a * n3 + c] = ld(s->A + 2 * ((3 * i + a) * n3 + c));
        return;
    }
    for (int64_t j = 0; j < s->n; ++j) {
        cplx G[3][3];
        src_entry(s, i, j, G);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) R[a * n3 + 3 * j + b] = G[a][b];
    }
}

static void src_col(const block_src* s, int64_t j, cplx* C /* 3m x 3 row-major */)
{
    const int64_t n3 = 3 * s->n;
    if (s->kind == 0) {
        for (int64_t r = 0; r < 3 * s->m; ++r)
            for (int b = 0; b < 3; ++b) C[3 * r + b] = ld(s->A + 2 * (r * n3 + 3 * j + b));
        return;
    }
    for (int64_t i = 0; i < s->m; ++i) {
        cplx G[3][3];
        src_entry(s, i, j, G);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) C[3 * (3 * i + a) + b] = G[a][b];
    }
}

/* Threshold below which a candidate pivot block counts as singular, relative
 * to the largest sigma_1 seen in the block's residual rows. */
#define ACA_SINGULAR_REL 1e-12

/* Runs the ACA; U (3m x k) and V (3n x k) col-major grow as needed.
 * Returns k (a multiple of 3).  pivots (optional, 2 per step) logs (i^, j^).
 * lost (optional): set to 1 when a row had to be retired for singular pivot
 * blocks although its residual was not negligible (largest sigma_1 of its
 * 3x3 blocks above eps times the largest sigma_1 seen): the vector ACA cannot
 * pivot such a row (every 3x3 block singular, e.g. coplanar T blocks), so the
 * approximation misses it. */
static int64_t aca_run(const block_src* s, double eps, cplx** Uout, cplx** Vout,
                       int64_t** pivlog, int* lost)
{
    if (lost) *lost = 0;
    const int64_t m = s->m, n = s->n, m3 = 3 * m, n3 = 3 * n;
    const int64_t kmax_steps = m < n ? m : n;
    int64_t cap = 8; /* steps of capacity */
    cplx* U = (cplx*)malloc((size_t)(m3 * 3 * cap) * sizeof(cplx));
    cplx* V = (cplx*)malloc((size_t)(n3 * 3 * cap) * sizeof(cplx));
    int64_t* piv = (int64_t*)malloc((size_t)(2 * cap) * sizeof(int64_t));
    char* used_row = (char*)calloc((size_t)m, 1);
    char* used_col = (char*)calloc((size_t)n, 1);
    cplx* R = (cplx*)malloc((size_t)(3 * n3) * sizeof(cplx));
    cplx* C = (cplx*)malloc((size_t)(m3 * 3) * sizeof(cplx));
    double* s3 = (double*)malloc((size_t)(m > n ? m : n) * sizeof(double));
    int64_t k = 0;          /* number of rank-3 steps taken */
    double normB2 = 0.0;    /* ||B_k||_F^2 */
    double sref = 0.0;      /* largest sigma_1 seen in a residual row */
    int64_t ihat = 0;       /* first row: the first point of tau (reading) */

    while (k < kmax_steps) {
        /* step 1: row block of the residual R_k(i^, :) = A(i^, :) - U(i^, :) V^H */
        src_row(s, ihat, R);
        for (int64_t l = 0; l < 3 * k; ++l)
            for (int a = 0; a < 3; ++a) {
                const cplx u = U[(3 * ihat + a) + l * m3];
                for (int64_t c = 0; c < n3; ++c) R[a * n3 + c] -= u * conj(V[c + l * n3]);
            }
        /* step 2: j^ = argmax sigma_3 of the 3x3 blocks R(i^, j), j unused */
        int64_t jhat = -1;
        double best = -1.0, rowmax = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            cplx B[3][3];
            double sv[3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) B[a][b] = R[a * n3 + 3 * j + b];
            sv3(B, sv);
            if (sv[0] > sref) sref = sv[0];
            if (sv[0] > rowmax) rowmax = sv[0];
            if (used_col[j]) continue;
            if (sv[2] > best) {
                best = sv[2];
                jhat = j;
            }
        }
        if (jhat < 0) break; /* every column used */
        if (best <= ACA_SINGULAR_REL * sref) {
            /* singular pivot: this row is exhausted; retry on the lowest unused row */
            if (lost && rowmax > eps * sref) *lost = 1;
            used_row[ihat] = 1;
            int64_t nxt = -1;
            for (int64_t i = 0; i < m; ++i)
                if (!used_row[i]) {
                    nxt = i;
                    break;
                }
            if (nxt < 0) break;
            ihat = nxt;
            continue;
        }
        cplx P[3][3], gam[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) P[a][b] = R[a * n3 + 3 * jhat + b];
        inv3(P, gam);
        /* step 3: column block R_k(:, j^) = A(:, j^) - U V(j^, :)^H */
        src_col(s, jhat, C);
        for (int64_t l = 0; l < 3 * k; ++l)
            for (int b = 0; b < 3; ++b) {
                const cplx vc = conj(V[(3 * jhat + b) + l * n3]);
                for (int64_t r = 0; r < m3; ++r) C[3 * r + b] -= U[r + l * m3] * vc;
            }
        /* step 4: next i^ = argmax sigma_3 of C(i, :), i unused, on the
         * column before the update of step 6 */
        used_row[ihat] = 1;
        used_col[jhat] = 1;
        int64_t inext = -1;
        double bestr = -1.0;
        for (int64_t i = 0; i < m; ++i) {
            if (used_row[i]) continue;
            cplx B[3][3];
            double sv[3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) B[a][b] = C[3 * (3 * i + a) + b];
            sv3(B, sv);
            if (sv[2] > bestr) {
                bestr = sv[2];
                inext = i;
            }
        }
        /* step 5: U_{k+1} = R_k(:, j^) gamma, V_{k+1} = R_k(i^, :)^H */
        if (k == cap) {
            cap *= 2;
            U = (cplx*)realloc(U, (size_t)(m3 * 3 * cap) * sizeof(cplx));
            V = (cplx*)realloc(V, (size_t)(n3 * 3 * cap) * sizeof(cplx));
            piv = (int64_t*)realloc(piv, (size_t)(2 * cap) * sizeof(int64_t));
        }
        cplx* Un = U + (3 * k) * m3;
        cplx* Vn = V + (3 * k) * n3;
        for (int b = 0; b < 3; ++b)
            for (int64_t r = 0; r < m3; ++r) {
                cplx acc = 0.0;
                for (int a = 0; a < 3; ++a) acc += C[3 * r + a] * gam[a][b];
                Un[r + b * m3] = acc;
            }
        for (int a = 0; a < 3; ++a)
            for (int64_t c = 0; c < n3; ++c) Vn[c + a * n3] = conj(R[a * n3 + c]);
        piv[2 * k] = ihat;
        piv[2 * k + 1] = jhat;
        /* step 6: B_{k+1} = B_k + U_{k+1} V_{k+1}^H, and
         * ||B_{k+1}||^2 = ||B_k||^2 + 2 Re <B_k, dB> + ||dB||^2 with
         * <u_p v_p^H, u_q v_q^H> = (u_p^H u_q)(v_q^H v_p). */
        cplx cross = 0.0;
        for (int64_t p = 0; p < 3 * k; ++p)
            for (int q = 0; q < 3; ++q) {
                cplx uu = 0.0, vv = 0.0;
                for (int64_t r = 0; r < m3; ++r) uu += conj(U[r + p * m3]) * Un[r + q * m3];
                for (int64_t c = 0; c < n3; ++c) vv += conj(Vn[c + q * n3]) * V[c + p * n3];
                cross += uu * vv;
            }
        double dB2 = 0.0;
        for (int q = 0; q < 3; ++q)
            for (int q2 = 0; q2 < 3; ++q2) {
                cplx uu = 0.0, vv = 0.0;
                for (int64_t r = 0; r < m3; ++r) uu += conj(Un[r + q * m3]) * Un[r + q2 * m3];
                for (int64_t c = 0; c < n3; ++c) vv += conj(Vn[c + q2 * n3]) * Vn[c + q * n3];
                dB2 += creal(uu * vv);
            }
        normB2 = normB2 + 2.0 * creal(cross) + dB2;
        k++;
        /* Eq. stop_part, read for the rank-3 step as ||B_{k+1} - B_k||_F
         * <= eps ||B_{k+1}||_F (the paper's ||u|| ||v|| is ||u v^*||_F). */
        if (sqrt(dB2) <= eps * sqrt(normB2 > 0.0 ? normB2 : 0.0)) break;
        if (inext < 0) break;
        ihat = inext;
    }
    free(used_row);
    free(used_col);
    free(R);
    free(C);
    free(s3);
    *Uout = U;
    *Vout = V;
    if (pivlog)
        *pivlog = piv;
    else
        free(piv);
    return 3 * k;
}

int64_t or_aca_dense(const double* A, int64_t m, int64_t n, double eps, int64_t kcap, double* U,
                     double* V, int64_t* pivots)
{
    block_src s = {0};
    s.kind = 0;
    s.m = m;
    s.n = n;
    s.A = A;
    cplx *Uc, *Vc;
    int64_t* pv;
    const int64_t k = aca_run(&s, eps, &Uc, &Vc, &pv, NULL);
    int64_t ret = k;
    if (k > kcap) {
        ret = -1;
    } else {
        for (int64_t i = 0; i < 3 * m * k; ++i) st(U + 2 * i, Uc[i]);
        for (int64_t i = 0; i < 3 * n * k; ++i) st(V + 2 * i, Vc[i]);
        if (pivots)
            for (int64_t i = 0; i < 2 * (k / 3); ++i) pivots[i] = pv[i];
    }
    free(Uc);
    free(Vc);
    free(pv);
    return ret;
}

/* ======================================================================
 * Recompression (Sec. 3.2): U V^H = Q_U R_U R_V^H Q_V^H; SVD R_U R_V^H = P S L^H;
 * U' = Q_U P S^{1/2}, V' = Q_V L S^{1/2}, truncated with eps_ACA.  Reading:
 * keep the smallest r' with (sum_{i>r'} s_i^2)^{1/2} <= eps (sum s_i^2)^{1/2}
 * (the Frobenius norm of the ACA stopping test); r' = 0 is allowed.
 * ====================================================================== */
static int64_t recompress(const cplx* U, const cplx* V, int64_t M, int64_t N, int64_t k,
                          double eps, cplx** U2, cplx** V2, double* svals_out)
{
    if (k == 0) {
        *U2 = NULL;
        *V2 = NULL;
        return 0;
    }
    cplx* QU = (cplx*)malloc((size_t)(M * k) * sizeof(cplx));
    cplx* QV = (cplx*)malloc((size_t)(N * k) * sizeof(cplx));
    cplx* RU = (cplx*)malloc((size_t)(k * k) * sizeof(cplx));
    cplx* RV = (cplx*)malloc((size_t)(k * k) * sizeof(cplx));
    qr_householder(U, M, k, QU, RU);
    qr_householder(V, N, k, QV, RV);
    cplx* W = (cplx*)malloc((size_t)(k * k) * sizeof(cplx));
    /* W = R_U R_V^H */
    for (int64_t c = 0; c < k; ++c)
        for (int64_t r = 0; r < k; ++r) {
            cplx acc = 0.0;
            for (int64_t t = 0; t < k; ++t) acc += RU[r + t * k] * conj(RV[c + t * k]);
            W[r + c * k] = acc;
        }
    double* s = (double*)malloc((size_t)k * sizeof(double));
    cplx* L = (cplx*)malloc((size_t)(k * k) * sizeof(cplx));
    svd_jacobi(W, k, k, s, L); /* W now holds P S (columns P_i s_i) */
    double tot = 0.0;
    for (int64_t i = 0; i < k; ++i) tot += s[i] * s[i];
    int64_t r = k;
    {
        double tail = 0.0; /* sum_{i >= r} s_i^2, grown from the end */
        for (int64_t i = k - 1; i >= 0; --i) {
            if (sqrt(tail + s[i] * s[i]) <= eps * sqrt(tot))
                tail += s[i] * s[i], r = i;
            else
                break;
        }
    }
    if (svals_out)
        for (int64_t i = 0; i < k; ++i) svals_out[i] = s[i];
    cplx* Uo = r ? (cplx*)malloc((size_t)(M * r) * sizeof(cplx)) : NULL;
    cplx* Vo = r ? (cplx*)malloc((size_t)(N * r) * sizeof(cplx)) : NULL;
    for (int64_t j = 0; j < r; ++j) {
        const double sq = sqrt(s[j]);
        /* P_j = W_j / s_j, so Q_U P_j s_j^{1/2} = Q_U W_j / s_j^{1/2} */
        for (int64_t row = 0; row < M; ++row) {
            cplx acc = 0.0;
            for (int64_t t = 0; t < k; ++t) acc += QU[row + t * M] * W[t + j * k];
            Uo[row + j * M] = acc / sq;
        }
        for (int64_t row = 0; row < N; ++row) {
            cplx acc = 0.0;
            for (int64_t t = 0; t < k; ++t) acc += QV[row + t * N] * L[t + j * k];
            Vo[row + j * N] = acc * sq;
        }
    }
    free(QU);
    free(QV);
    free(RU);
    free(RV);
    free(W);
    free(s);
    free(L);
    *U2 = Uo;
    *V2 = Vo;
    return r;
}

int64_t or_recompress(const double* U, const double* V, int64_t M, int64_t N, int64_t k,
                      double eps, double* U2, double* V2, double* svals)
{
    cplx* u = (cplx*)malloc((size_t)(M * k + 1) * sizeof(cplx));
    cplx* v = (cplx*)malloc((size_t)(N * k + 1) * sizeof(cplx));
    for (int64_t i = 0; i < M * k; ++i) u[i] = ld(U + 2 * i);
    for (int64_t i = 0; i < N * k; ++i) v[i] = ld(V + 2 * i);
    cplx *uo, *vo;
    const int64_t r = recompress(u, v, M, N, k, eps, &uo, &vo, svals);
    for (int64_t i = 0; i < M * r; ++i) st(U2 + 2 * i, uo[i]);
    for (int64_t i = 0; i < N * r; ++i) st(V2 + 2 * i, vo[i]);
    free(u);
    free(v);
    free(uo);
    free(vo);
    return r;
}

/* ======================================================================
 * Randomized SVD (the remark closing Sec. 2.3, which prefers the randomized
 * SVD of Liberty, Woolfe, Martinsson, Rokhlin & Tygert 2007 to the vector ACA
 * for blocks whose 3x3 sub-blocks are all singular).  For a block A (3m x 3n):
 *   1. draw a Gaussian test matrix Omega (3n x l) and sketch Y = A Omega;
 *   2. Q = an orthonormal basis of range(Y) (Householder QR);
 *   3. B = Q^H A, so that A ~ Q B;
 * the number of samples l doubles until p further probe columns w certify
 * the range error; the factors (U, V) = (Q, B^H) then go through the
 * recompression of Sec. 3.2 (QR, SVD of the core, truncation).
 * Readings (the remark names the method only):
 *   Omega(j, c) is a complex normal number with E|w|^2 = 1, made by the
 *     Box-Muller transform from two uniforms of the splitmix64 generator
 *     (Steele, Lea & Flood 2014) applied to a counter (j, c) under a key made
 *     from the block's first row and column point in tree order, so that any
 *     implementation of the same published definitions draws the same matrix;
 *   l starts at 64 and doubles, up to min(3m, 3n, 768);
 *   the range is accepted when the mean over p = 8 probes of
 *     |(I - Q Q^H) A w|^2 is at most (eps/4)^2 ||A||_F^2; since
 *     E|(I - Q Q^H) A w|^2 = ||(I - Q Q^H) A||_F^2, the range error is then
 *     below eps/2 ||A||_F with high probability, and the recompression
 *     truncates with eps sqrt(3)/2: the two errors are orthogonal, so the
 *     total stays below eps ||A||_F.
 * ====================================================================== */
#define RSVD_L0 64
#define RSVD_P 8
#define RSVD_LMAX 768
#define RSVD_CSTRIDE 1024 /* counter of Omega(j, c) = j * RSVD_CSTRIDE + c */

static uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static cplx rsvd_gauss(uint64_t key, uint64_t ctr)
{
    const uint64_t a = splitmix64(key ^ splitmix64(2 * ctr));
    const uint64_t b = splitmix64(key ^ splitmix64(2 * ctr + 1));
    const double u1 = (double)((a >> 11) + 1) * 0x1.0p-53; /* (0, 1] */
    const double u2 = (double)(b >> 11) * 0x1.0p-53;       /* [0, 1) */
    const double r = sqrt(-log(u1)); /* sqrt(-2 ln u1) times the 1/sqrt(2) of E|w|^2 = 1 */
    const double th = 2.0 * M_PI * u2;
    return r * cos(th) + I * (r * sin(th));
}

uint64_t or_splitmix64(uint64_t z) { return splitmix64(z); }

uint64_t or_rsvd_key(int64_t tau_begin, int64_t sigma_begin)
{
    return splitmix64(((uint64_t)tau_begin << 32) ^ (uint64_t)sigma_begin);
}

void or_gauss(uint64_t key, uint64_t ctr, double* out2) { st(out2, rsvd_gauss(key, ctr)); }

/* Runs steps 1-3 on the block of source s; returns l, with U = Q (3m x l) and
 * V = B^H (3n x l) col-major in *Uout, *Vout.  *ok = 0 if l reached its cap
 * without the probes' certificate. */
static int64_t rsvd_run(const block_src* s, double eps, uint64_t key, cplx** Uout, cplx** Vout,
                        int* ok)
{
    const int64_t M = 3 * s->m, N = 3 * s->n;
    cplx* A = (cplx*)malloc((size_t)(M * N) * sizeof(cplx));
    cplx* C = (cplx*)malloc((size_t)(3 * M) * sizeof(cplx));
    for (int64_t j = 0; j < s->n; ++j) {
        src_col(s, j, C); /* 3m x 3 row-major */
        for (int64_t r = 0; r < M; ++r)
            for (int b = 0; b < 3; ++b) A[r + (3 * j + b) * M] = C[3 * r + b];
    }
    free(C);
    double anorm2 = 0.0;
    for (int64_t e = 0; e < M * N; ++e) anorm2 += abs2(A[e]);
    int64_t lmax = M < N ? M : N;
    if (lmax > RSVD_LMAX) lmax = RSVD_LMAX;
    int64_t l = lmax < RSVD_L0 ? lmax : RSVD_L0;
    cplx *Y = NULL, *Q = NULL, *R = NULL;
    *ok = 0;
    for (;;) {
        const int64_t L = l + RSVD_P;
        Y = (cplx*)malloc((size_t)(M * L) * sizeof(cplx));
        for (int64_t c = 0; c < L; ++c)
            for (int64_t r = 0; r < M; ++r) Y[r + c * M] = 0.0;
        for (int64_t j = 0; j < N; ++j)
            for (int64_t c = 0; c < L; ++c) {
                const cplx w = rsvd_gauss(key, (uint64_t)j * RSVD_CSTRIDE + (uint64_t)c);
                for (int64_t r = 0; r < M; ++r) Y[r + c * M] += A[r + j * M] * w;
            }
        Q = (cplx*)malloc((size_t)(M * l) * sizeof(cplx));
        R = (cplx*)malloc((size_t)(l * l) * sizeof(cplx));
        qr_householder(Y, M, l, Q, R);
        double est = 0.0;
        for (int64_t c = l; c < L; ++c) { /* |y - Q Q^H y|^2 of the probe column */
            const cplx* y = Y + c * M;
            cplx* z = (cplx*)malloc((size_t)M * sizeof(cplx));
            for (int64_t r = 0; r < M; ++r) z[r] = y[r];
            for (int64_t t = 0; t < l; ++t) {
                cplx d = 0.0;
                for (int64_t r = 0; r < M; ++r) d += conj(Q[r + t * M]) * y[r];
                for (int64_t r = 0; r < M; ++r) z[r] -= Q[r + t * M] * d;
            }
            for (int64_t r = 0; r < M; ++r) est += abs2(z[r]);
            free(z);
        }
        est /= RSVD_P;
        free(Y);
        free(R);
        if (est <= (eps / 4) * (eps / 4) * anorm2) *ok = 1;
        if (*ok || l == lmax) break;
        free(Q);
        l = 2 * l < lmax ? 2 * l : lmax;
    }
    cplx* V = (cplx*)malloc((size_t)(N * l) * sizeof(cplx));
    for (int64_t c = 0; c < l; ++c)
        for (int64_t j = 0; j < N; ++j) {
            cplx acc = 0.0;
            for (int64_t r = 0; r < M; ++r) acc += conj(A[r + j * M]) * Q[r + c * M];
            V[j + c * N] = acc;
        }
    free(A);
    *Uout = Q;
    *Vout = V;
    return l;
}

int64_t or_rsvd_dense(const double* A, int64_t m, int64_t n, double eps, uint64_t key,
                      int64_t lcap, double* U, double* V, int* ok)
{
    block_src src = {0};
    src.kind = 0;
    src.m = m;
    src.n = n;
    src.A = A;
    cplx *u, *v;
    const int64_t l = rsvd_run(&src, eps, key, &u, &v, ok);
    if (l > lcap) {
        free(u);
        free(v);
        return -1;
    }
    for (int64_t i = 0; i < 3 * m * l; ++i) st(U + 2 * i, u[i]);
    for (int64_t i = 0; i < 3 * n * l; ++i) st(V + 2 * i, v[i]);
    free(u);
    free(v);
    return l;
}

/* ======================================================================
 * H-matrix: tree + partition + per-block data (Sec. 2, Sec. 3.1).
 * ====================================================================== */
struct or_hmat {
    or_problem pb;
    int64_t nc;
    int64_t* perm;
    or_cluster* cl;
    int64_t ncl;
    or_block* blk;
    int64_t nb;
    int64_t* rank_aca;
    int64_t* rank;
    cplx** D;  /* dense data, or U */
    cplx** V;  /* low-rank V */
    char* method; /* admissible blocks: 0 vector ACA, 1 randomized SVD */
    char* built;
    double build_s;
};

static double now_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

or_hmat* or_hmat_build(const or_problem* pb, const double* pts, const double* nrm, int64_t nc,
                       double eps, double eta, int64_t leaf, int recompress_on,
                       int64_t sample_stride, int nthreads)
{
    const double t0 = now_s();
    or_hmat* h = (or_hmat*)calloc(1, sizeof(or_hmat));
    h->pb = *pb;
    h->nc = nc;
    h->perm = (int64_t*)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int64_t));
    h->cl = (or_cluster*)malloc((size_t)(2 * nc + 1) * sizeof(or_cluster));
    h->ncl = or_tree_build(pts, nc, leaf, h->perm, h->cl);
    h->nb = or_partition(h->cl, h->ncl, eta, NULL);
    h->blk = (or_block*)malloc((size_t)(h->nb + 1) * sizeof(or_block));
    or_partition(h->cl, h->ncl, eta, h->blk);
    h->rank_aca = (int64_t*)calloc((size_t)(h->nb + 1), sizeof(int64_t));
    h->rank = (int64_t*)calloc((size_t)(h->nb + 1), sizeof(int64_t));
    h->D = (cplx**)calloc((size_t)(h->nb + 1), sizeof(cplx*));
    h->V = (cplx**)calloc((size_t)(h->nb + 1), sizeof(cplx*));
    h->built = (char*)calloc((size_t)(h->nb + 1), 1);
    h->method = (char*)calloc((size_t)(h->nb + 1), 1);
    if (sample_stride < 1) sample_stride = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t b = 0; b < h->nb; ++b) {
        if (b % sample_stride) continue;
        const or_cluster* t = &h->cl[h->blk[b].tau];
        const or_cluster* s = &h->cl[h->blk[b].sigma];
        const int64_t m = t->end - t->begin, n = s->end - s->begin;
        if (!h->blk[b].admissible) {
            /* dense near-field block: A(tau, sigma), col-major 3m x 3n */
            cplx* D = (cplx*)malloc((size_t)(9 * m * n) * sizeof(cplx));
            for (int64_t j = 0; j < n; ++j)
                for (int64_t i = 0; i < m; ++i) {
                    cplx G[3][3];
                    entry_block(pb, pts, nrm, h->perm[t->begin + i], h->perm[s->begin + j], G);
                    for (int a = 0; a < 3; ++a)
                        for (int c = 0; c < 3; ++c) D[(3 * i + a) + (3 * j + c) * (3 * m)] = G[a][c];
                }
            h->D[b] = D;
        } else {
            block_src src = {0};
            src.kind = 1;
            src.m = m;
            src.n = n;
            src.pb = pb;
            src.pts = pts;
            src.nrm = nrm;
            src.rows = h->perm + t->begin;
            src.cols = h->perm + s->begin;
            cplx *U, *V;
            int lost = 0;
            const int64_t k = aca_run(&src, eps, &U, &V, NULL, &lost);
            h->rank_aca[b] = k;
            if (lost) {
                /* rows the vector ACA cannot pivot (every 3x3 block singular):
                 * the randomized SVD (remark of Sec. 2.3) compresses the block */
                free(U);
                free(V);
                int ok = 0;
                const int64_t l = rsvd_run(&src, eps, or_rsvd_key(t->begin, s->begin), &U, &V, &ok);
                h->rank_aca[b] = l;
                h->method[b] = ok ? 1 : 2;
                if (recompress_on) {
                    cplx *U2, *V2;
                    const int64_t r = recompress(U, V, 3 * m, 3 * n, l, eps * sqrt(3.0) / 2, &U2, &V2, NULL);
                    free(U);
                    free(V);
                    h->D[b] = U2;
                    h->V[b] = V2;
                    h->rank[b] = r;
                } else {
                    h->D[b] = U;
                    h->V[b] = V;
                    h->rank[b] = l;
                }
            } else if (recompress_on) {
                cplx *U2, *V2;
                const int64_t r = recompress(U, V, 3 * m, 3 * n, k, eps, &U2, &V2, NULL);
                free(U);
                free(V);
                h->D[b] = U2;
                h->V[b] = V2;
                h->rank[b] = r;
            } else {
                h->D[b] = U;
                h->V[b] = V;
                h->rank[b] = k;
            }
        }
        h->built[b] = 1;
    }
    h->build_s = now_s() - t0;
    return h;
}

void or_hmat_free(or_hmat* h)
{
    if (!h) return;
    for (int64_t b = 0; b < h->nb; ++b) {
        free(h->D[b]);
        free(h->V[b]);
    }
    free(h->D);
    free(h->V);
    free(h->built);
    free(h->method);
    free(h->rank);
    free(h->rank_aca);
    free(h->blk);
    free(h->cl);
    free(h->perm);
    free(h);
}

void or_hmat_block_methods(const or_hmat* h, int32_t* out)
{
    for (int64_t b = 0; b < h->nb; ++b) out[b] = h->method[b];
}

int64_t or_hmat_nclusters(const or_hmat* h) { return h->ncl; }
void or_hmat_clusters(const or_hmat* h, or_cluster* out)
{
    memcpy(out, h->cl, (size_t)h->ncl * sizeof(or_cluster));
}
void or_hmat_perm(const or_hmat* h, int64_t* perm)
{
    memcpy(perm, h->perm, (size_t)h->nc * sizeof(int64_t));
}
int64_t or_hmat_nblocks(const or_hmat* h) { return h->nb; }
void or_hmat_blocks(const or_hmat* h, or_block* out, int64_t* rank_aca, int64_t* rank)
{
    for (int64_t b = 0; b < h->nb; ++b) {
        if (out) out[b] = h->blk[b];
        if (rank_aca) rank_aca[b] = h->built[b] ? h->rank_aca[b] : -1;
        if (rank) rank[b] = h->built[b] ? h->rank[b] : -1;
    }
}
double or_hmat_build_seconds(const or_hmat* h) { return h->build_s; }

void or_hmat_block_data(const or_hmat* h, int64_t b, double* D_or_U, double* V)
{
    const or_cluster* t = &h->cl[h->blk[b].tau];
    const or_cluster* s = &h->cl[h->blk[b].sigma];
    const int64_t m3 = 3 * (t->end - t->begin), n3 = 3 * (s->end - s->begin);
    if (!h->built[b]) return;
    if (!h->blk[b].admissible) {
        for (int64_t i = 0; i < m3 * n3; ++i) st(D_or_U + 2 * i, h->D[b][i]);
        return;
    }
    const int64_t r = h->rank[b];
    for (int64_t i = 0; i < m3 * r; ++i) st(D_or_U + 2 * i, h->D[b][i]);
    for (int64_t i = 0; i < n3 * r; ++i) st(V + 2 * i, h->V[b][i]);
}

/* Sec. 3.1: y = sum over P^non-ad of A_b x_sigma + sum over P^ad of U (V^H x_sigma).
 * x, y are complex128 in the original point order; blocks live in tree order. */
static void hmat_apply(const or_hmat* h, const cplx* x, cplx* y)
{
    const int64_t N = 3 * h->nc;
    cplx* xp = (cplx*)malloc((size_t)(N + 1) * sizeof(cplx));
    cplx* yp = (cplx*)calloc((size_t)(N + 1), sizeof(cplx));
    for (int64_t p = 0; p < h->nc; ++p)
        for (int a = 0; a < 3; ++a) xp[3 * p + a] = x[3 * h->perm[p] + a];
    for (int64_t b = 0; b < h->nb; ++b) {
        if (!h->built[b]) continue;
        const or_cluster* t = &h->cl[h->blk[b].tau];
        const or_cluster* s = &h->cl[h->blk[b].sigma];
        const int64_t m3 = 3 * (t->end - t->begin), n3 = 3 * (s->end - s->begin);
        const cplx* xs = xp + 3 * s->begin;
        cplx* yt = yp + 3 * t->begin;
        if (!h->blk[b].admissible) {
            const cplx* D = h->D[b];
            for (int64_t c = 0; c < n3; ++c)
                for (int64_t r = 0; r < m3; ++r) yt[r] += D[r + c * m3] * xs[c];
        } else {
            const int64_t k = h->rank[b];
            const cplx* U = h->D[b];
            const cplx* V = h->V[b];
            for (int64_t l = 0; l < k; ++l) {
                cplx tl = 0.0;
                for (int64_t c = 0; c < n3; ++c) tl += conj(V[c + l * n3]) * xs[c];
                for (int64_t r = 0; r < m3; ++r) yt[r] += U[r + l * m3] * tl;
            }
        }
    }
    for (int64_t p = 0; p < h->nc; ++p)
        for (int a = 0; a < 3; ++a) y[3 * h->perm[p] + a] = yp[3 * p + a];
    free(xp);
    free(yp);
}

void or_hmat_matvec(const or_hmat* h, const double* x, double* y)
{
    hmat_apply(h, (const cplx*)x, (cplx*)y);
}

/* ======================================================================
 * Two clouds: targets X (rows, the collocation points x_i) and sources Y
 * (columns, the points y_j with their normals and weights), each with its
 * own cluster tree (Sec. 2.1); the partition pairs a cluster of X with a
 * cluster of Y by the same recursion and admissibility test as the square
 * case.  Blocks are dense or compressed exactly as there (vector ACA,
 * randomized SVD for unpivotable rows, recompression).
 * ====================================================================== */
static void part_rec2(const or_cluster* clX, const or_cluster* clY, double eta, int64_t t, int64_t s,
                      or_block* out, int64_t* nb)
{
    const int adm = or_admissible_box(clX[t].lo, clX[t].hi, clY[s].lo, clY[s].hi, eta);
    if (adm || clX[t].is_leaf || clY[s].is_leaf) {
        if (out) {
            out[*nb].tau = t;
            out[*nb].sigma = s;
            out[*nb].admissible = adm;
            out[*nb].pad_ = 0;
        }
        (*nb)++;
        return;
    }
    const int64_t tc[2] = {clX[t].child0, clX[t].child1};
    const int64_t sc[2] = {clY[s].child0, clY[s].child1};
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) part_rec2(clX, clY, eta, tc[u], sc[v], out, nb);
}

int64_t or_partition2(const or_cluster* clX, int64_t nclX, const or_cluster* clY, int64_t nclY, double eta,
                      or_block* out)
{
    if (nclX == 0 || nclY == 0) return 0;
    int64_t nb = 0;
    part_rec2(clX, clY, eta, 0, 0, out, &nb);
    return nb;
}

struct or_hmat2 {
    or_problem pb;
    int64_t nx, ny;
    int64_t *permX, *permY;
    or_cluster *clX, *clY;
    int64_t nclX, nclY;
    or_block* blk;
    int64_t nb;
    int64_t *rank_aca, *rank;
    cplx** D; /* dense data, or U */
    cplx** V;
};

or_hmat2* or_hmat2_build(const or_problem* pb, const double* X, int64_t nx, const double* Y, int64_t ny,
                         const double* nrmY, double eps, double eta, int64_t leaf, int nthreads)
{
    or_hmat2* h = (or_hmat2*)calloc(1, sizeof(or_hmat2));
    h->pb = *pb;
    h->nx = nx;
    h->ny = ny;
    h->permX = (int64_t*)malloc((size_t)(nx > 0 ? nx : 1) * sizeof(int64_t));
    h->permY = (int64_t*)malloc((size_t)(ny > 0 ? ny : 1) * sizeof(int64_t));
    h->clX = (or_cluster*)malloc((size_t)(2 * nx + 1) * sizeof(or_cluster));
    h->clY = (or_cluster*)malloc((size_t)(2 * ny + 1) * sizeof(or_cluster));
    h->nclX = or_tree_build(X, nx, leaf, h->permX, h->clX);
    h->nclY = or_tree_build(Y, ny, leaf, h->permY, h->clY);
    h->nb = or_partition2(h->clX, h->nclX, h->clY, h->nclY, eta, NULL);
    h->blk = (or_block*)malloc((size_t)(h->nb + 1) * sizeof(or_block));
    or_partition2(h->clX, h->nclX, h->clY, h->nclY, eta, h->blk);
    h->rank_aca = (int64_t*)calloc((size_t)(h->nb + 1), sizeof(int64_t));
    h->rank = (int64_t*)calloc((size_t)(h->nb + 1), sizeof(int64_t));
    h->D = (cplx**)calloc((size_t)(h->nb + 1), sizeof(cplx*));
    h->V = (cplx**)calloc((size_t)(h->nb + 1), sizeof(cplx*));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t b = 0; b < h->nb; ++b) {
        const or_cluster* t = &h->clX[h->blk[b].tau];
        const or_cluster* s = &h->clY[h->blk[b].sigma];
        const int64_t m = t->end - t->begin, n = s->end - s->begin;
        if (!h->blk[b].admissible) {
            cplx* D = (cplx*)malloc((size_t)(9 * m * n + 1) * sizeof(cplx));
            for (int64_t j = 0; j < n; ++j)
                for (int64_t i = 0; i < m; ++i) {
                    cplx G[3][3];
                    entry_block2(pb, X, Y, nrmY, h->permX[t->begin + i], h->permY[s->begin + j], G);
                    for (int a = 0; a < 3; ++a)
                        for (int c = 0; c < 3; ++c) D[(3 * i + a) + (3 * j + c) * (3 * m)] = G[a][c];
                }
            h->D[b] = D;
            continue;
        }
        block_src src = {0};
        src.kind = 1;
        src.m = m;
        src.n = n;
        src.pb = pb;
        src.pts = X;
        src.pts_y = Y;
        src.nrm_y = nrmY;
        src.rows = h->permX + t->begin;
        src.cols = h->permY + s->begin;
        cplx *U, *V;
        int lost = 0;
        int64_t k = aca_run(&src, eps, &U, &V, NULL, &lost);
        double eps_r = eps;
        if (lost) { /* rows the vector ACA cannot pivot: the randomized SVD */
            free(U);
            free(V);
            int ok = 0;
            k = rsvd_run(&src, eps, or_rsvd_key(t->begin, s->begin), &U, &V, &ok);
            eps_r = eps * sqrt(3.0) / 2;
        }
        h->rank_aca[b] = k;
        cplx *U2, *V2;
        h->rank[b] = recompress(U, V, 3 * m, 3 * n, k, eps_r, &U2, &V2, NULL);
        free(U);
        free(V);
        h->D[b] = U2;
        h->V[b] = V2;
    }
    return h;
}

void or_hmat2_free(or_hmat2* h)
{
    if (!h) return;
    for (int64_t b = 0; b < h->nb; ++b) {
        free(h->D[b]);
        free(h->V[b]);
    }
    free(h->D);
    free(h->V);
    free(h->rank);
    free(h->rank_aca);
    free(h->blk);
    free(h->clX);
    free(h->clY);
    free(h->permX);
    free(h->permY);
    free(h);
}

int64_t or_hmat2_nblocks(const or_hmat2* h) { return h->nb; }
void or_hmat2_blocks(const or_hmat2* h, or_block* out, int64_t* rank)
{
    for (int64_t b = 0; b < h->nb; ++b) {
        if (out) out[b] = h->blk[b];
        if (rank) rank[b] = h->rank[b];
    }
}
void or_hmat2_clusters(const or_hmat2* h, or_cluster* clX, or_cluster* clY)
{
    if (clX) memcpy(clX, h->clX, (size_t)h->nclX * sizeof(or_cluster));
    if (clY) memcpy(clY, h->clY, (size_t)h->nclY * sizeof(or_cluster));
}
int64_t or_hmat2_nclusters(const or_hmat2* h, int side) { return side ? h->nclY : h->nclX; }

/* y = A_H x: x on the sources (3 ny, original order), y on the targets (3 nx). */
void or_hmat2_matvec(const or_hmat2* h, const double* xd, double* yd)
{
    const cplx* x = (const cplx*)xd;
    cplx* y = (cplx*)yd;
    cplx* xp = (cplx*)malloc((size_t)(3 * h->ny + 1) * sizeof(cplx));
    cplx* yp = (cplx*)calloc((size_t)(3 * h->nx + 1), sizeof(cplx));
    for (int64_t p = 0; p < h->ny; ++p)
        for (int a = 0; a < 3; ++a) xp[3 * p + a] = x[3 * h->permY[p] + a];
    for (int64_t b = 0; b < h->nb; ++b) {
        const or_cluster* t = &h->clX[h->blk[b].tau];
        const or_cluster* s = &h->clY[h->blk[b].sigma];
        const int64_t m3 = 3 * (t->end - t->begin), n3 = 3 * (s->end - s->begin);
        const cplx* xs = xp + 3 * s->begin;
        cplx* yt = yp + 3 * t->begin;
        if (!h->blk[b].admissible) {
            const cplx* D = h->D[b];
            for (int64_t c = 0; c < n3; ++c)
                for (int64_t r = 0; r < m3; ++r) yt[r] += D[r + c * m3] * xs[c];
        } else {
            const cplx* U = h->D[b];
            const cplx* V = h->V[b];
            for (int64_t l = 0; l < h->rank[b]; ++l) {
                cplx tl = 0.0;
                for (int64_t c = 0; c < n3; ++c) tl += conj(V[c + l * n3]) * xs[c];
                for (int64_t r = 0; r < m3; ++r) yt[r] += U[r + l * m3] * tl;
            }
        }
    }
    for (int64_t p = 0; p < h->nx; ++p)
        for (int a = 0; a < 3; ++a) y[3 * h->permX[p] + a] = yp[3 * p + a];
    free(xp);
    free(yp);
}

/* ======================================================================
 * Restarted GMRES(m): Arnoldi with modified Gram-Schmidt, complex Givens
 * rotations, x0 = 0; converged when the true residual ||b - A x||/||b|| <= tol
 * (checked at each restart; inside a cycle the Givens estimate decides when
 * to restart early).
 * ====================================================================== */
typedef void (*apply_fn)(const void* ctx, const cplx* x, cplx* y);

static double vnorm(const cplx* v, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += abs2(v[i]);
    return sqrt(s);
}

static int gmres(apply_fn A, const void* ctx, int64_t n, const cplx* b, cplx* x, int m,
                 double tol, int maxit, int* iters, double* relres)
{
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    const double bn = vnorm(b, n);
    *iters = 0;
    if (bn == 0.0) {
        *relres = 0.0;
        return 0;
    }
    cplx* Vb = (cplx*)malloc((size_t)(n * (m + 1)) * sizeof(cplx));
    cplx* H = (cplx*)calloc((size_t)((m + 1) * m), sizeof(cplx)); /* H[i + j*(m+1)] */
    cplx* cs = (cplx*)malloc((size_t)m * sizeof(cplx));
    cplx* sn = (cplx*)malloc((size_t)m * sizeof(cplx));
    cplx* g = (cplx*)malloc((size_t)(m + 1) * sizeof(cplx));
    cplx* yv = (cplx*)malloc((size_t)m * sizeof(cplx));
    cplx* w = (cplx*)malloc((size_t)n * sizeof(cplx));
    int status = 1;
    for (;;) {
        A(ctx, x, w);
        for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
        const double beta = vnorm(w, n);
        *relres = beta / bn;
        if (*relres <= tol) {
            status = 0;
            break;
        }
        if (*iters >= maxit) break;
        for (int64_t i = 0; i < n; ++i) Vb[i] = w[i] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int jend = 0;
        for (int j = 0; j < m; ++j) {
            A(ctx, Vb + (int64_t)j * n, w);
            (*iters)++;
            for (int i = 0; i <= j; ++i) {
                cplx hij = 0.0;
                for (int64_t q = 0; q < n; ++q) hij += conj(Vb[q + (int64_t)i * n]) * w[q];
                H[i + j * (m + 1)] = hij;
                for (int64_t q = 0; q < n; ++q) w[q] -= hij * Vb[q + (int64_t)i * n];
            }
            const double hn = vnorm(w, n);
            H[(j + 1) + j * (m + 1)] = hn;
            if (hn > 0.0)
                for (int64_t q = 0; q < n; ++q) Vb[q + (int64_t)(j + 1) * n] = w[q] / hn;
            for (int i = 0; i < j; ++i) { /* previous rotations */
                const cplx h0 = H[i + j * (m + 1)], h1 = H[(i + 1) + j * (m + 1)];
                H[i + j * (m + 1)] = cs[i] * h0 + sn[i] * h1;
                H[(i + 1) + j * (m + 1)] = -conj(sn[i]) * h0 + cs[i] * h1;
            }
            const cplx a = H[j + j * (m + 1)], bb = H[(j + 1) + j * (m + 1)];
            const double nu = sqrt(abs2(a) + abs2(bb));
            if (cabs(a) == 0.0) {
                cs[j] = 0.0;
                sn[j] = 1.0;
            } else {
                cs[j] = cabs(a) / nu;
                sn[j] = (a / cabs(a)) * conj(bb) / nu;
            }
            H[j + j * (m + 1)] = cs[j] * a + sn[j] * bb;
            H[(j + 1) + j * (m + 1)] = 0.0;
            const cplx g0 = g[j];
            g[j] = cs[j] * g0;
            g[j + 1] = -conj(sn[j]) * g0;
            jend = j + 1;
            if (cabs(g[j + 1]) / bn <= tol || *iters >= maxit || hn == 0.0) break;
        }
        for (int i = jend - 1; i >= 0; --i) { /* back substitution */
            cplx acc = g[i];
            for (int q = i + 1; q < jend; ++q) acc -= H[i + q * (m + 1)] * yv[q];
            yv[i] = acc / H[i + i * (m + 1)];
        }
        for (int i = 0; i < jend; ++i)
            for (int64_t q = 0; q < n; ++q) x[q] += yv[i] * Vb[q + (int64_t)i * n];
    }
    free(Vb);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(yv);
    free(w);
    return status;
}

static void apply_hmat(const void* ctx, const cplx* x, cplx* y)
{
    hmat_apply((const or_hmat*)ctx, x, y);
}

typedef struct {
    const cplx* A;
    int64_t n;
} dense_ctx;

static void apply_dense(const void* ctx, const cplx* x, cplx* y)
{
    const dense_ctx* d = (const dense_ctx*)ctx;
    for (int64_t i = 0; i < d->n; ++i) {
        cplx acc = 0.0;
        for (int64_t j = 0; j < d->n; ++j) acc += d->A[i * d->n + j] * x[j];
        y[i] = acc;
    }
}

int or_gmres_hmat(const or_hmat* h, const double* b, double* x, int restart, double tol,
                  int maxit, int* iters, double* relres)
{
    return gmres(apply_hmat, h, 3 * h->nc, (const cplx*)b, (cplx*)x, restart, tol, maxit, iters,
                 relres);
}

int or_gmres_dense(const double* A, int64_t n, const double* b, double* x, int restart,
                   double tol, int maxit, int* iters, double* relres)
{
    dense_ctx d = {(const cplx*)A, n};
    return gmres(apply_dense, &d, n, (const cplx*)b, (cplx*)x, restart, tol, maxit, iters, relres);
}

/* ======================================================================
 * H-LU factorisation and direct solver (Sec. 3.2, "H-LU factorization and
 * direct solver").  The H-matrix is copied into its block tree (the recursion
 * of the partition: a node is a dense block, a low-rank block U V^H, or the
 * 2 x 2 block matrix of its children) and factorised recursively on 2 x 2
 * block matrices in the four steps of Sec. 3.2:
 *   1. A11 = L11 U11 (recursion; a dense diagonal leaf is factorised in place);
 *   2. U12 = L11^{-1} A12;
 *   3. L21 = A21 U11^{-1};
 *   4. A22 <- A22 - L21 U12, then A22 = L22 U22 (recursion).
 * The update of step 4 (A''' = A + A' A'', the "27 cases") is formed in the
 * format of the target block: into a dense target as a dense update, into a
 * subdivided target child by child, into a low-rank target as a low-rank
 * update [U, -U_p] [V, V_p]^H recompressed (Sec. 3.2: QR of both factors, SVD
 * of R_U R_V^H) with eps_LU; a product with a low-rank factor stays factored
 * (A U_b) V_b^H or U_a (B^H V_a)^H, the product of two dense or subdivided
 * blocks is formed densely.  L (unit lower) and U share the tree in place.
 * Readings (the paper leaves them open): no pivoting; a dense update of a
 * low-rank target enters as [U, -P] [V, I]^H before the recompression.
 * ====================================================================== */
typedef struct hnode {
    int type;              /* 0 dense, 1 low rank, 2 subdivided */
    int64_t m, n;          /* rows, columns (DOFs) */
    cplx* D;               /* dense: m x n col-major */
    cplx *U, *V;           /* low rank: U (m x k), V (n x k); block = U V^H */
    int64_t k;
    struct hnode* ch[4];   /* (t0 s0), (t0 s1), (t1 s0), (t1 s1) */
    int64_t m0, n0;        /* rows of t0, columns of s0 (subdivided) */
} hnode;

struct or_hlu {
    int64_t nc;
    int64_t* perm;
    hnode* root;
    double eps;
    double seconds;
};

static hnode* hn_build(const or_hmat* h, int64_t t, int64_t s, int64_t* bi, double eta)
{
    const or_cluster* cl = h->cl;
    hnode* x = (hnode*)calloc(1, sizeof(hnode));
    x->m = 3 * (cl[t].end - cl[t].begin);
    x->n = 3 * (cl[s].end - cl[s].begin);
    const int adm = or_admissible_box(cl[t].lo, cl[t].hi, cl[s].lo, cl[s].hi, eta);
    if (adm || cl[t].is_leaf || cl[s].is_leaf) { /* a leaf of the partition: the next block */
        const int64_t b = (*bi)++;
        if (b >= h->nb || h->blk[b].tau != t || h->blk[b].sigma != s) { /* not the partition's order */
            x->type = 0;
            x->D = (cplx*)calloc((size_t)(x->m * x->n + 1), sizeof(cplx));
            *bi = h->nb + 1;
            return x;
        }
        if (h->blk[b].admissible) {
            x->type = 1;
            x->k = h->rank[b];
            x->U = (cplx*)malloc((size_t)(x->m * x->k + 1) * sizeof(cplx));
            x->V = (cplx*)malloc((size_t)(x->n * x->k + 1) * sizeof(cplx));
            memcpy(x->U, h->D[b], (size_t)(x->m * x->k) * sizeof(cplx));
            memcpy(x->V, h->V[b], (size_t)(x->n * x->k) * sizeof(cplx));
        } else {
            x->type = 0;
            x->D = (cplx*)malloc((size_t)(x->m * x->n) * sizeof(cplx));
            memcpy(x->D, h->D[b], (size_t)(x->m * x->n) * sizeof(cplx));
        }
        return x;
    }
    x->type = 2;
    const int64_t tc[2] = {cl[t].child0, cl[t].child1};
    const int64_t sc[2] = {cl[s].child0, cl[s].child1};
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) x->ch[2 * u + v] = hn_build(h, tc[u], sc[v], bi, eta);
    x->m0 = x->ch[0]->m;
    x->n0 = x->ch[0]->n;
    return x;
}

static void hn_free(hnode* x)
{
    if (!x) return;
    for (int q = 0; q < 4; ++q) hn_free(x->ch[q]);
    free(x->D);
    free(x->U);
    free(x->V);
    free(x);
}

/* Y (m x c, ld ldy) += alpha * op(x) X (X: n x c or m x c for the adjoint), op = x or x^H */
static void hn_apply(const hnode* x, int adj, const cplx* X, int64_t ldx, cplx* Y, int64_t ldy,
                     int64_t c, cplx alpha)
{
    const int64_t rows = adj ? x->n : x->m, cols = adj ? x->m : x->n;
    if (x->type == 0) {
        for (int64_t j = 0; j < c; ++j)
            for (int64_t q = 0; q < cols; ++q) {
                const cplx xv = alpha * X[q + j * ldx];
                if (xv == 0.0) continue;
                for (int64_t r = 0; r < rows; ++r)
                    Y[r + j * ldy] += (adj ? conj(x->D[q + r * x->m]) : x->D[r + q * x->m]) * xv;
            }
        return;
    }
    if (x->type == 1) { /* U V^H X, or V U^H X */
        const cplx* A = adj ? x->U : x->V; /* contracted with X */
        const cplx* B = adj ? x->V : x->U; /* spans the result */
        const int64_t la = adj ? x->m : x->n, lb = adj ? x->n : x->m;
        for (int64_t j = 0; j < c; ++j)
            for (int64_t l = 0; l < x->k; ++l) {
                cplx t = 0.0;
                for (int64_t q = 0; q < la; ++q) t += conj(A[q + l * la]) * X[q + j * ldx];
                t *= alpha;
                for (int64_t r = 0; r < lb; ++r) Y[r + j * ldy] += B[r + l * lb] * t;
            }
        return;
    }
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const hnode* y = x->ch[2 * u + v];
            const int64_t ro = u ? x->m0 : 0, co = v ? x->n0 : 0;
            if (!adj)
                hn_apply(y, 0, X + co, ldx, Y + ro, ldy, c, alpha);
            else
                hn_apply(y, 1, X + ro, ldx, Y + co, ldy, c, alpha);
        }
}

/* B (m x c) <- L^{-1} B, L the unit lower factor of the diagonal node x */
static void hn_solve_l(const hnode* x, cplx* B, int64_t ldb, int64_t c)
{
    if (x->type == 0) {
        for (int64_t j = 0; j < c; ++j)
            for (int64_t r = 0; r < x->m; ++r) {
                cplx acc = B[r + j * ldb];
                for (int64_t q = 0; q < r; ++q) acc -= x->D[r + q * x->m] * B[q + j * ldb];
                B[r + j * ldb] = acc;
            }
        return;
    }
    hn_solve_l(x->ch[0], B, ldb, c);
    hn_apply(x->ch[2], 0, B, ldb, B + x->m0, ldb, c, -1.0);
    hn_solve_l(x->ch[3], B + x->m0, ldb, c);
}

/* B (m x c) <- U^{-1} B, U the upper factor of the diagonal node x */
static void hn_solve_u(const hnode* x, cplx* B, int64_t ldb, int64_t c)
{
    if (x->type == 0) {
        for (int64_t j = 0; j < c; ++j)
            for (int64_t r = x->m - 1; r >= 0; --r) {
                cplx acc = B[r + j * ldb];
                for (int64_t q = r + 1; q < x->m; ++q) acc -= x->D[r + q * x->m] * B[q + j * ldb];
                B[r + j * ldb] = acc / x->D[r + r * x->m];
            }
        return;
    }
    hn_solve_u(x->ch[3], B + x->m0, ldb, c);
    hn_apply(x->ch[1], 0, B + x->m0, ldb, B, ldb, c, -1.0);
    hn_solve_u(x->ch[0], B, ldb, c);
}

/* B (n x c) <- U^{-H} B (solves U^H Y = B: forward substitution with U^H) */
static void hn_solve_uh(const hnode* x, cplx* B, int64_t ldb, int64_t c)
{
    if (x->type == 0) {
        for (int64_t j = 0; j < c; ++j)
            for (int64_t r = 0; r < x->m; ++r) {
                cplx acc = B[r + j * ldb];
                for (int64_t q = 0; q < r; ++q) acc -= conj(x->D[q + r * x->m]) * B[q + j * ldb];
                B[r + j * ldb] = acc / conj(x->D[r + r * x->m]);
            }
        return;
    }
    hn_solve_uh(x->ch[0], B, ldb, c);
    hn_apply(x->ch[1], 1, B, ldb, B + x->n0, ldb, c, -1.0);
    hn_solve_uh(x->ch[3], B + x->n0, ldb, c);
}

/* x += alpha Up Vp^H (Up: m x k, Vp: n x k, leading dimensions lu, lv) */
static void hn_add_lr(hnode* x, const cplx* Up, int64_t lu, const cplx* Vp, int64_t lv, int64_t k,
                      cplx alpha, double eps)
{
    if (k == 0) return;
    if (x->type == 0) {
        for (int64_t l = 0; l < k; ++l)
            for (int64_t j = 0; j < x->n; ++j) {
                const cplx v = alpha * conj(Vp[j + l * lv]);
                for (int64_t i = 0; i < x->m; ++i) x->D[i + j * x->m] += Up[i + l * lu] * v;
            }
        return;
    }
    if (x->type == 2) {
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v)
                hn_add_lr(x->ch[2 * u + v], Up + (u ? x->m0 : 0), lu, Vp + (v ? x->n0 : 0), lv, k,
                          alpha, eps);
        return;
    }
    /* low-rank target: [U, alpha Up] [V, Vp]^H, recompressed with eps_LU */
    int64_t K = x->k + k;
    cplx* U2 = (cplx*)malloc((size_t)(x->m * K + 1) * sizeof(cplx));
    cplx* V2 = (cplx*)malloc((size_t)(x->n * K + 1) * sizeof(cplx));
    memcpy(U2, x->U, (size_t)(x->m * x->k) * sizeof(cplx));
    memcpy(V2, x->V, (size_t)(x->n * x->k) * sizeof(cplx));
    for (int64_t l = 0; l < k; ++l) {
        for (int64_t i = 0; i < x->m; ++i) U2[i + (x->k + l) * x->m] = alpha * Up[i + l * lu];
        for (int64_t j = 0; j < x->n; ++j) V2[j + (x->k + l) * x->n] = Vp[j + l * lv];
    }
    if (K > x->m || K > x->n) {
        /* more columns than the block's smaller side: the sum densely, then
         * factored as D I^H (or I D^H) with min(m, n) columns */
        cplx* Dn = (cplx*)calloc((size_t)(x->m * x->n + 1), sizeof(cplx));
        for (int64_t l = 0; l < K; ++l)
            for (int64_t j = 0; j < x->n; ++j) {
                const cplx v = conj(V2[j + l * x->n]);
                for (int64_t i = 0; i < x->m; ++i) Dn[i + j * x->m] += U2[i + l * x->m] * v;
            }
        free(U2);
        free(V2);
        if (x->m >= x->n) {
            K = x->n;
            U2 = Dn;
            V2 = (cplx*)calloc((size_t)(x->n * x->n + 1), sizeof(cplx));
            for (int64_t j = 0; j < x->n; ++j) V2[j + j * x->n] = 1.0;
        } else {
            K = x->m;
            U2 = (cplx*)calloc((size_t)(x->m * x->m + 1), sizeof(cplx));
            for (int64_t i = 0; i < x->m; ++i) U2[i + i * x->m] = 1.0;
            V2 = (cplx*)malloc((size_t)(x->n * x->m + 1) * sizeof(cplx));
            for (int64_t i = 0; i < x->m; ++i)
                for (int64_t j = 0; j < x->n; ++j) V2[j + i * x->n] = conj(Dn[i + j * x->m]);
            free(Dn);
        }
    }
    free(x->U);
    free(x->V);
    cplx *U3, *V3;
    x->k = recompress(U2, V2, x->m, x->n, K, eps, &U3, &V3, NULL);
    free(U2);
    free(V2);
    x->U = U3 ? U3 : (cplx*)calloc(1, sizeof(cplx));
    x->V = V3 ? V3 : (cplx*)calloc(1, sizeof(cplx));
}

/* x += alpha P (P: m x n dense, leading dimension lp) */
static void hn_add_dense(hnode* x, const cplx* P, int64_t lp, cplx alpha, double eps)
{
    if (x->type == 0) {
        for (int64_t j = 0; j < x->n; ++j)
            for (int64_t i = 0; i < x->m; ++i) x->D[i + j * x->m] += alpha * P[i + j * lp];
        return;
    }
    if (x->type == 2) {
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v)
                hn_add_dense(x->ch[2 * u + v], P + (u ? x->m0 : 0) + (v ? x->n0 : 0) * lp, lp, alpha, eps);
        return;
    }
    /* low-rank target: alpha P = (alpha P) I^H */
    cplx* Id = (cplx*)calloc((size_t)(x->n * x->n + 1), sizeof(cplx));
    for (int64_t j = 0; j < x->n; ++j) Id[j + j * x->n] = 1.0;
    hn_add_lr(x, P, lp, Id, x->n, x->n, alpha, eps);
    free(Id);
}

/* C -= A B  (A: m x l, B: l x n nodes) */
static void hn_gemm_sub(hnode* C, const hnode* A, const hnode* B, double eps)
{
    if (C->type == 2 && A->type == 2 && B->type == 2) {
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v)
                for (int w = 0; w < 2; ++w)
                    hn_gemm_sub(C->ch[2 * u + v], A->ch[2 * u + w], B->ch[2 * w + v], eps);
        return;
    }
    if (B->type == 1) { /* A (U_b V_b^H) = (A U_b) V_b^H */
        cplx* AU = (cplx*)calloc((size_t)(A->m * B->k + 1), sizeof(cplx));
        hn_apply(A, 0, B->U, B->m, AU, A->m, B->k, 1.0);
        hn_add_lr(C, AU, A->m, B->V, B->n, B->k, -1.0, eps);
        free(AU);
        return;
    }
    if (A->type == 1) { /* (U_a V_a^H) B = U_a (B^H V_a)^H */
        cplx* BV = (cplx*)calloc((size_t)(B->n * A->k + 1), sizeof(cplx));
        hn_apply(B, 1, A->V, A->n, BV, B->n, A->k, 1.0);
        hn_add_lr(C, A->U, A->m, BV, B->n, A->k, -1.0, eps);
        free(BV);
        return;
    }
    /* dense or subdivided operands: the product densely, P = A B */
    cplx* Bd = (cplx*)calloc((size_t)(B->m * B->n + 1), sizeof(cplx));
    cplx* Id = (cplx*)calloc((size_t)(B->n * B->n + 1), sizeof(cplx));
    for (int64_t j = 0; j < B->n; ++j) Id[j + j * B->n] = 1.0;
    hn_apply(B, 0, Id, B->n, Bd, B->m, B->n, 1.0); /* B densely */
    free(Id);
    cplx* P = (cplx*)calloc((size_t)(A->m * B->n + 1), sizeof(cplx));
    hn_apply(A, 0, Bd, B->m, P, A->m, B->n, 1.0);
    free(Bd);
    hn_add_dense(C, P, A->m, -1.0, eps);
    free(P);
}

/* X <- L^{-1} X for the node X (rows of the diagonal node L) */
static void hn_trsm_l(const hnode* L, hnode* X, double eps)
{
    if (X->type == 0) {
        hn_solve_l(L, X->D, X->m, X->n);
    } else if (X->type == 1) {
        hn_solve_l(L, X->U, X->m, X->k);
    } else { /* X subdivided, so is L (same row cluster) */
        for (int v = 0; v < 2; ++v) {
            hn_trsm_l(L->ch[0], X->ch[v], eps);
            hn_gemm_sub(X->ch[2 + v], L->ch[2], X->ch[v], eps);
            hn_trsm_l(L->ch[3], X->ch[2 + v], eps);
        }
    }
}

/* X <- X U^{-1} for the node X (columns of the diagonal node U) */
static void hn_trsm_u(const hnode* Uf, hnode* X, double eps)
{
    if (X->type == 0) { /* X^H <- U^{-H} X^H */
        cplx* T = (cplx*)malloc((size_t)(X->m * X->n + 1) * sizeof(cplx));
        for (int64_t i = 0; i < X->m; ++i)
            for (int64_t j = 0; j < X->n; ++j) T[j + i * X->n] = conj(X->D[i + j * X->m]);
        hn_solve_uh(Uf, T, X->n, X->m);
        for (int64_t i = 0; i < X->m; ++i)
            for (int64_t j = 0; j < X->n; ++j) X->D[i + j * X->m] = conj(T[j + i * X->n]);
        free(T);
    } else if (X->type == 1) { /* U_x (V_x^H U^{-1}) = U_x (U^{-H} V_x)^H */
        hn_solve_uh(Uf, X->V, X->n, X->k);
    } else {
        for (int u = 0; u < 2; ++u) {
            hn_trsm_u(Uf->ch[0], X->ch[2 * u], eps);
            hn_gemm_sub(X->ch[2 * u + 1], X->ch[2 * u], Uf->ch[1], eps);
            hn_trsm_u(Uf->ch[3], X->ch[2 * u + 1], eps);
        }
    }
}

static int hn_lu(hnode* x, double eps)
{
    if (x->type == 0) { /* dense LU without pivoting, in place */
        for (int64_t p = 0; p < x->m; ++p) {
            const cplx piv = x->D[p + p * x->m];
            if (piv == 0.0) return 1;
            for (int64_t r = p + 1; r < x->m; ++r) x->D[r + p * x->m] /= piv;
            for (int64_t c = p + 1; c < x->n; ++c) {
                const cplx u = x->D[p + c * x->m];
                for (int64_t r = p + 1; r < x->m; ++r) x->D[r + c * x->m] -= x->D[r + p * x->m] * u;
            }
        }
        return 0;
    }
    if (hn_lu(x->ch[0], eps)) return 1;            /* 1. A11 = L11 U11 */
    hn_trsm_l(x->ch[0], x->ch[1], eps);            /* 2. U12 = L11^{-1} A12 */
    hn_trsm_u(x->ch[0], x->ch[2], eps);            /* 3. L21 = A21 U11^{-1} */
    hn_gemm_sub(x->ch[3], x->ch[2], x->ch[1], eps); /* 4. A22 - L21 U12 ... */
    return hn_lu(x->ch[3], eps);                   /*    = L22 U22 */
}

static int64_t hn_stored(const hnode* x)
{
    if (x->type == 0) return x->m * x->n;
    if (x->type == 1) return (x->m + x->n) * x->k;
    int64_t s = 0;
    for (int q = 0; q < 4; ++q) s += hn_stored(x->ch[q]);
    return s;
}

or_hlu* or_hlu_factor(const or_hmat* h, double eta, double eps_lu, int* status)
{
    const double t0 = now_s();
    or_hlu* f = (or_hlu*)calloc(1, sizeof(or_hlu));
    f->nc = h->nc;
    f->perm = (int64_t*)malloc((size_t)(h->nc + 1) * sizeof(int64_t));
    memcpy(f->perm, h->perm, (size_t)h->nc * sizeof(int64_t));
    int64_t bi = 0;
    f->root = hn_build(h, 0, 0, &bi, eta);
    f->eps = eps_lu;
    *status = (bi == h->nb) ? hn_lu(f->root, eps_lu) : 2; /* 1: zero pivot, 2: partition mismatch */
    f->seconds = now_s() - t0;
    return f;
}

void or_hlu_free(or_hlu* f)
{
    if (!f) return;
    hn_free(f->root);
    free(f->perm);
    free(f);
}

/* x = U^{-1} L^{-1} b, vectors in the original point order */
void or_hlu_solve(const or_hlu* f, const double* b, double* x)
{
    const int64_t N = 3 * f->nc;
    cplx* y = (cplx*)malloc((size_t)(N + 1) * sizeof(cplx));
    for (int64_t p = 0; p < f->nc; ++p)
        for (int a = 0; a < 3; ++a) y[3 * p + a] = ld(b + 2 * (3 * f->perm[p] + a));
    hn_solve_l(f->root, y, N, 1);
    hn_solve_u(f->root, y, N, 1);
    for (int64_t p = 0; p < f->nc; ++p)
        for (int a = 0; a < 3; ++a) st(x + 2 * (3 * f->perm[p] + a), y[3 * p + a]);
    free(y);
}

/* L (unit lower) and U as dense N x N col-major matrices in tree order */
void or_hlu_dense(const or_hlu* f, double* L, double* U)
{
    const int64_t N = 3 * f->nc;
    cplx* Mi = (cplx*)calloc((size_t)(N * N + 1), sizeof(cplx)); /* L^{-1}, then U^{-1} */
    cplx* F = (cplx*)calloc((size_t)(N * N + 1), sizeof(cplx));  /* L, then U */
    for (int64_t j = 0; j < N; ++j) Mi[j + j * N] = 1.0;
    hn_solve_l(f->root, Mi, N, N); /* Mi = L^{-1}, unit lower triangular */
    for (int64_t j = 0; j < N; ++j) /* L = Mi^{-1}: forward substitution, column by column */
        for (int64_t r = j; r < N; ++r) {
            cplx acc = (r == j) ? 1.0 : 0.0;
            for (int64_t q = j; q < r; ++q) acc -= Mi[r + q * N] * F[q + j * N];
            F[r + j * N] = acc;
        }
    for (int64_t e = 0; e < N * N; ++e) st(L + 2 * e, F[e]);
    memset(Mi, 0, (size_t)(N * N) * sizeof(cplx));
    memset(F, 0, (size_t)(N * N) * sizeof(cplx));
    for (int64_t j = 0; j < N; ++j) Mi[j + j * N] = 1.0;
    hn_solve_u(f->root, Mi, N, N); /* Mi = U^{-1}, upper triangular */
    for (int64_t j = 0; j < N; ++j) /* U = Mi^{-1}: backward substitution, column by column */
        for (int64_t r = j; r >= 0; --r) {
            cplx acc = (r == j) ? 1.0 : 0.0;
            for (int64_t q = r + 1; q <= j; ++q) acc -= Mi[r + q * N] * F[q + j * N];
            F[r + j * N] = acc / Mi[r + r * N];
        }
    for (int64_t e = 0; e < N * N; ++e) st(U + 2 * e, F[e]);
    free(Mi);
    free(F);
}

double or_hlu_seconds(const or_hlu* f) { return f->seconds; }
int64_t or_hlu_stored(const or_hlu* f) { return hn_stored(f->root); }

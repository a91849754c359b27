/*
 * mlbm_oracle.c -- plain, slow FP64 CPU oracle of the meshless lattice Boltzmann method
 * (MLBM) studied in Strzelczyk & Matyka, "Study of the convergence of the Meshless Lattice
 * Boltzmann Method in Taylor-Green and annular channel flows" (arXiv 2306.01525).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline leg
 * of bench.py may load this library.  It shares no code, header, table or helper with the
 * GPU library, and the GPU library never calls it.
 *
 * Every function is double precision with scalar loops in the order the paper states the
 * method; no blocking, fusion or reordering beyond the paper's own steps.  Each function
 * names the section / equation / algorithm it follows.
 *
 * Array conventions: node fields are SoA, field[c * n + i]; stencil and weight tables are
 * [dir][j][i] = tab[(dir * K + j) * n + i].  Indices are int64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 9

/* D2Q9 lattice directions e_k, k = 0..8, in the order of Sec. 2.1. */
static const int orc_ex[ORC_Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int orc_ey[ORC_Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* Lattice weights omega_k of Sec. 2.1. */
static double orc_omega(int k)
{
    if (k == 0) return 4.0 / 9.0;
    if (k <= 4) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

/* Lattice speed of sound squared, c_s = 1/sqrt(3) (Sec. 2.1). */
static const double orc_cs2 = 1.0 / 3.0;

int orc_abi_version(void) { return 1; }

/* Export the velocity set and weights so tests can check the tables against Sec. 2.1. */
void orc_d2q9(int *ex, int *ey, double *omega)
{
    for (int k = 0; k < ORC_Q; ++k) {
        ex[k] = orc_ex[k];
        ey[k] = orc_ey[k];
        omega[k] = orc_omega(k);
    }
}

/* Opposite direction k' with e_k' = -e_k (Sec. 2.1), found by search, not by table. */
int orc_opposite(int k)
{
    for (int kk = 0; kk < ORC_Q; ++kk)
        if (orc_ex[kk] == -orc_ex[k] && orc_ey[kk] == -orc_ey[k]) return kk;
    return -1;
}

/* Equilibrium distribution, eq. (feq) of Sec. 2.1, in lattice units (c_k = e_k). */
double orc_feq(int k, double rho, double ux, double uy)
{
    double cu = orc_ex[k] * ux + orc_ey[k] * uy;
    double uu = ux * ux + uy * uy;
    return orc_omega(k) * rho *
           (1.0 + cu / orc_cs2 + (cu * cu) / (2.0 * orc_cs2 * orc_cs2) - uu / (2.0 * orc_cs2));
}

/* Macroscopic density and velocity, eq. (macro_var); the sums run over all nine
 * populations (the printed lower index 1 is read as the first direction, k = 0). */
void orc_moments(const double *f, double *rho, double *ux, double *uy)
{
    double r = 0.0, mx = 0.0, my = 0.0;
    for (int k = 0; k < ORC_Q; ++k) {
        r += f[k];
        mx += f[k] * orc_ex[k];
        my += f[k] * orc_ey[k];
    }
    *rho = r;
    *ux = mx / r;
    *uy = my / r;
}

/* BGK collision, eq. (LBM_collision), plus the body-force term omega_k e_k.g / c_s^2 of the
 * annular-channel section (Sec. 3).  f and fpost hold the nine populations of one node. */
void orc_collide(const double *f, double tau, double gx, double gy, double *fpost)
{
    double rho, ux, uy;
    orc_moments(f, &rho, &ux, &uy);
    for (int k = 0; k < ORC_Q; ++k) {
        double feq = orc_feq(k, rho, ux, uy);
        double force = orc_omega(k) * (orc_ex[k] * gx + orc_ey[k] * gy) / orc_cs2;
        fpost[k] = f[k] - (f[k] - feq) / tau + force;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Geometry: periodic minimum image (Sec. 3, periodic stencil search).                  */
/* ------------------------------------------------------------------------------------ */

/* Shortest periodic representative of a coordinate difference; L <= 0 means no wrap. */
static double orc_wrap(double d, double L)
{
    if (L > 0.0) d -= L * round(d / L);
    return d;
}

static double orc_dist2(double ax, double ay, double bx, double by, double lx, double ly)
{
    double dx = orc_wrap(ax - bx, lx);
    double dy = orc_wrap(ay - by, ly);
    return dx * dx + dy * dy;
}

/* The K nodes closest to point (qx, qy) by brute force over all n nodes, ordered by
 * (squared distance, node index) ascending.  For a query at node i the node itself comes
 * first, as the stencil centre of Sec. 2.2.  Returns 0, or -1 if K > n. */
int orc_knn(const double *x, const double *y, int64_t n, double qx, double qy, int K,
            double lx, double ly, int64_t *out)
{
    if (K < 1 || K > n) return -1;
    double *bd = (double *)malloc(sizeof(double) * (size_t)K);
    int cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        double d2 = orc_dist2(x[j], y[j], qx, qy, lx, ly);
        /* insertion into the sorted list of the best K (ties: lower index first, which
         * the ascending scan over j gives by inserting after equal keys) */
        if (cnt == K && d2 >= bd[K - 1]) continue;
        int pos = (cnt < K) ? cnt : K - 1;
        while (pos > 0 && bd[pos - 1] > d2) {
            bd[pos] = bd[pos - 1];
            out[pos] = out[pos - 1];
            --pos;
        }
        bd[pos] = d2;
        out[pos] = j;
        if (cnt < K) ++cnt;
    }
    free(bd);
    return 0;
}

/* Own K-nearest-neighbour stencil X^L of every node (Sec. 2.2): stencil[j * n + i]. */
int orc_build_stencils(const double *x, const double *y, int64_t n, int K, double lx,
                       double ly, int64_t *stencil)
{
    if (K < 1 || K > n) return -1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
        if (orc_knn(x, y, n, x[i], y[i], K, lx, ly, tmp) != 0) err = -1;
        for (int j = 0; j < K; ++j) stencil[(int64_t)j * n + i] = tmp[j];
        free(tmp);
    }
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* RBF interpolation, Sec. 2.2 and 2.3                                                  */
/* ------------------------------------------------------------------------------------ */

/* Number of monomials of total degree <= deg (the sets P_i of eq. (poly_sets)). */
int orc_num_monomials(int dim, int deg)
{
    if (deg < 0) return 0;
    if (dim == 1) return deg + 1;
    return (deg + 1) * (deg + 2) / 2;
}

static double orc_ipow(double v, int p)
{
    double r = 1.0;
    for (int i = 0; i < p; ++i) r *= v;
    return r;
}

/* Monomials x^a y^b, a + b <= deg, by total degree and then by decreasing power of x, the
 * order in which eq. (poly_sets) lists P_2 and P_4.  dim == 1 gives 1, x, ..., x^deg. */
void orc_monomials(int dim, int deg, double x, double y, double *out)
{
    int c = 0;
    for (int t = 0; t <= deg; ++t) {
        if (dim == 1) {
            out[c++] = orc_ipow(x, t);
            continue;
        }
        for (int b = 0; b <= t; ++b) out[c++] = orc_ipow(x, t - b) * orc_ipow(y, b);
    }
}

/* Cubic polyharmonic spline phi(r) = r^3 (Sec. 2.3). */
static double orc_phi(double r) { return r * r * r; }

/* Solve A z = b (A n x n row-major, both overwritten) by Gaussian elimination with
 * partial pivoting, i.e. the LU factorisation with row pivoting the paper names in
 * Sec. 2.3, applied to one right-hand side.  Returns -1 if a pivot falls below
 * 1e-14 times the largest |A| entry. */
static int orc_lu_solve(double *A, double *b, int n, double *z)
{
    double amax = 0.0;
    for (int i = 0; i < n * n; ++i) amax = fmax(amax, fabs(A[i]));
    for (int p = 0; p < n; ++p) {
        int piv = p;
        double best = fabs(A[p * n + p]);
        for (int r = p + 1; r < n; ++r)
            if (fabs(A[r * n + p]) > best) {
                best = fabs(A[r * n + p]);
                piv = r;
            }
        if (!(best > 1e-14 * amax)) return -1;
        if (piv != p) {
            for (int c = 0; c < n; ++c) {
                double t = A[p * n + c];
                A[p * n + c] = A[piv * n + c];
                A[piv * n + c] = t;
            }
            double t = b[p];
            b[p] = b[piv];
            b[piv] = t;
        }
        for (int r = p + 1; r < n; ++r) {
            double l = A[r * n + p] / A[p * n + p];
            A[r * n + p] = l;
            for (int c = p + 1; c < n; ++c) A[r * n + c] -= l * A[p * n + c];
            b[r] -= l * b[p];
        }
    }
    for (int p = n - 1; p >= 0; --p) {
        double s = b[p];
        for (int c = p + 1; c < n; ++c) s -= A[p * n + c] * z[c];
        z[p] = s / A[p * n + p];
    }
    return 0;
}

/* Shape vector w_L(x) of eq. (shape_vector): w = Phi_L^{-1} phi_L(x), keeping the first
 * N_L entries.  (px, py) are the stencil members relative to the stencil centre, (qx, qy)
 * the evaluation point relative to the same centre.  Coordinates are divided by the
 * stencil radius s = max_j |p_j| before Phi_L is assembled (eq. (rbf_interp_set_augmented));
 * with phi = r^3 and a full polynomial space of total degree <= deg the shape vector is
 * unchanged by this scaling in exact arithmetic.  dim 1 uses py = qy = 0 and monomials
 * of x only.  Returns 0, -1 if Phi_L is numerically singular, -2 on bad sizes. */
int orc_shape_vector(int dim, int K, int deg, const double *px, const double *py, double qx,
                     double qy, double *w)
{
    int m = orc_num_monomials(dim, deg);
    int n = K + m;
    if (K < 1 || m > K || (dim != 1 && dim != 2)) return -2;
    double s = 0.0;
    for (int j = 0; j < K; ++j) {
        double yy = (dim == 2) ? py[j] : 0.0;
        s = fmax(s, sqrt(px[j] * px[j] + yy * yy));
    }
    if (s == 0.0) s = 1.0;
    double *A = (double *)calloc((size_t)n * n, sizeof(double));
    double *b = (double *)calloc((size_t)n, sizeof(double));
    double *z = (double *)calloc((size_t)n, sizeof(double));
    double *ma = (double *)calloc((size_t)m, sizeof(double));
    double *tx = (double *)calloc((size_t)K, sizeof(double));
    double *ty = (double *)calloc((size_t)K, sizeof(double));
    for (int j = 0; j < K; ++j) {
        tx[j] = px[j] / s;
        ty[j] = (dim == 2) ? py[j] / s : 0.0;
    }
    double sqx = qx / s, sqy = (dim == 2) ? qy / s : 0.0;
    /* R_L block: phi(|x_a - x_c|) */
    for (int a = 0; a < K; ++a)
        for (int c = 0; c < K; ++c) {
            double dx = tx[a] - tx[c], dy = ty[a] - ty[c];
            A[a * n + c] = orc_phi(sqrt(dx * dx + dy * dy));
        }
    /* P_L and P_L^T blocks; the lower-right block stays zero */
    for (int a = 0; a < K; ++a) {
        orc_monomials(dim, deg, tx[a], ty[a], ma);
        for (int l = 0; l < m; ++l) {
            A[a * n + K + l] = ma[l];
            A[(K + l) * n + a] = ma[l];
        }
    }
    /* right-hand side phi_L(x): radial functions then monomials at the evaluation point */
    for (int a = 0; a < K; ++a) {
        double dx = sqx - tx[a], dy = sqy - ty[a];
        b[a] = orc_phi(sqrt(dx * dx + dy * dy));
    }
    orc_monomials(dim, deg, sqx, sqy, ma);
    for (int l = 0; l < m; ++l) b[K + l] = ma[l];
    int rc = orc_lu_solve(A, b, n, z);
    if (rc == 0)
        for (int j = 0; j < K; ++j) w[j] = z[j];
    free(A);
    free(b);
    free(z);
    free(ma);
    free(tx);
    free(ty);
    return rc;
}

/* Stencils and shape vectors of the semi-Lagrangian streaming step (Sec. 2.3 and the
 * set-up loop of the appendix algorithm).  For every node i and direction k = 0..8 the
 * departure ("Lagrangian") point of population k is D_ik = x_i - e_k dx_ml.
 *   mode 0 ("own"):   the stencil is node i's own K-NN stencil;
 *   mode 1 ("paper"): the stencil is that of the Eulerian node closest to D_ik.
 * stencil[j*n+i] is the own K-NN table (orc_build_stencils).  Outputs:
 *   sidx[(k*K + j)*n + i]  member j of the stencil that interpolates direction k at node i
 *   W[(k*K + j)*n + i]     its shape-vector entry.
 * Returns 0, or the number of singular systems (negated) if any. */
int64_t orc_build_weights(const double *x, const double *y, int64_t n, int K, int deg,
                          double dx_ml, double lx, double ly, int mode,
                          const int64_t *stencil, int64_t *sidx, double *W)
{
    int64_t nbad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nbad)
    for (int64_t i = 0; i < n; ++i) {
        double *px = (double *)malloc(sizeof(double) * (size_t)K);
        double *py = (double *)malloc(sizeof(double) * (size_t)K);
        double *w = (double *)malloc(sizeof(double) * (size_t)K);
        for (int k = 0; k < ORC_Q; ++k) {
            double Dx = x[i] - orc_ex[k] * dx_ml;
            double Dy = y[i] - orc_ey[k] * dx_ml;
            int64_t L = i;
            if (mode == 1) {
                int64_t nn;
                orc_knn(x, y, n, Dx, Dy, 1, lx, ly, &nn);
                L = nn;
            }
            for (int j = 0; j < K; ++j) {
                int64_t s = stencil[(int64_t)j * n + L];
                px[j] = orc_wrap(x[s] - x[L], lx);
                py[j] = orc_wrap(y[s] - y[L], ly);
            }
            double qx = orc_wrap(Dx - x[L], lx);
            double qy = orc_wrap(Dy - y[L], ly);
            int rc = orc_shape_vector(2, K, deg, px, py, qx, qy, w);
            if (rc != 0) {
                nbad += 1;
                for (int j = 0; j < K; ++j) w[j] = 0.0;
            }
            for (int j = 0; j < K; ++j) {
                sidx[((int64_t)k * K + j) * n + i] = stencil[(int64_t)j * n + L];
                W[((int64_t)k * K + j) * n + i] = w[j];
            }
        }
        free(px);
        free(py);
        free(w);
    }
    return -nbad;
}

/* Stencils and shape vectors of ONE node i for all nine directions, found by brute force over
 * all n nodes (own stencil of i, or in mode 1 the stencil of the node nearest to each departure
 * point), exactly as orc_build_weights does for every node.  Outputs sidx[k*K + j] and
 * W[k*K + j], k = 0..8.  Returns the number of singular systems. */
int orc_node_weights(const double *x, const double *y, int64_t n, int64_t i, int K, int deg,
                     double dx_ml, double lx, double ly, int mode, int64_t *sidx, double *W)
{
    int nbad = 0;
    int64_t *st = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    double *px = (double *)malloc(sizeof(double) * (size_t)K);
    double *py = (double *)malloc(sizeof(double) * (size_t)K);
    for (int k = 0; k < ORC_Q; ++k) {
        double Dx = x[i] - orc_ex[k] * dx_ml;
        double Dy = y[i] - orc_ey[k] * dx_ml;
        int64_t L = i;
        if (mode == 1) orc_knn(x, y, n, Dx, Dy, 1, lx, ly, &L);
        orc_knn(x, y, n, x[L], y[L], K, lx, ly, st);
        for (int j = 0; j < K; ++j) {
            px[j] = orc_wrap(x[st[j]] - x[L], lx);
            py[j] = orc_wrap(y[st[j]] - y[L], ly);
        }
        double qx = orc_wrap(Dx - x[L], lx);
        double qy = orc_wrap(Dy - y[L], ly);
        if (orc_shape_vector(2, K, deg, px, py, qx, qy, W + (int64_t)k * K) != 0) {
            nbad += 1;
            for (int j = 0; j < K; ++j) W[(int64_t)k * K + j] = 0.0;
        }
        for (int j = 0; j < K; ++j) sidx[(int64_t)k * K + j] = st[j];
    }
    free(st);
    free(px);
    free(py);
    return nbad;
}

/* ------------------------------------------------------------------------------------ */
/* Annular channel (Sec. 3): body force and wall bounce-back                            */
/* ------------------------------------------------------------------------------------ */

/* Constant azimuthal acceleration g = (0, g) in polar coordinates, i.e.
 * g(x) = g (-sin(phi), cos(phi)) in Cartesian components (Sec. 3). */
void orc_azimuthal_force(const double *x, const double *y, int64_t n, double g, double *gx,
                         double *gy)
{
    for (int64_t i = 0; i < n; ++i) {
        double r = sqrt(x[i] * x[i] + y[i] * y[i]);
        gx[i] = (r > 0.0) ? -g * y[i] / r : 0.0;
        gy[i] = (r > 0.0) ? g * x[i] / r : 0.0;
    }
}

/* Unknown populations of the wall bounce-back (Sec. 3): bit k of mask[i] is set when the
 * departure point x_i - e_k dx_ml of population k lies outside the fluid annulus
 * r_in <= r <= r_out (relative tolerance 1e-12 on r^2). */
void orc_bounce_mask(const double *x, const double *y, int64_t n, double dx_ml, double r_in,
                     double r_out, uint16_t *mask)
{
    for (int64_t i = 0; i < n; ++i) {
        uint16_t m = 0;
        for (int k = 1; k < ORC_Q; ++k) {
            double Dx = x[i] - orc_ex[k] * dx_ml, Dy = y[i] - orc_ey[k] * dx_ml;
            double r2 = Dx * Dx + Dy * Dy;
            if (r2 < r_in * r_in * (1.0 - 1e-12) || r2 > r_out * r_out * (1.0 + 1e-12))
                m |= (uint16_t)(1u << k);
        }
        mask[i] = m;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Time loop (appendix algorithm)                                                        */
/* ------------------------------------------------------------------------------------ */

/* Initial populations: equilibrium at the initial macroscopic fields (Sec. 3 and the
 * set-up loop of the appendix algorithm). */
void orc_init_equilibrium(int64_t n, const double *rho, const double *ux, const double *uy,
                          double *f)
{
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < ORC_Q; ++k) f[(int64_t)k * n + i] = orc_feq(k, rho[i], ux[i], uy[i]);
}

/* One time step, COLLIDE then STREAM (Sec. 2.1 and the appendix algorithm), followed by
 * the wall bounce-back of Sec. 3:
 *   1. f_post = collide(f) at every node (force gx, gy may be NULL);
 *   2. f_k(i) <- sum_j W[k][j][i] f_post_k(sidx[k][j][i]) for k = 0..8;
 *   3. where bit k of mask[i] is set, f_k(i) <- the streamed f_k'(i) of step 2.
 * f_in and f_out are [9][n] and must differ; scratch holds [9][n] doubles. */
/* STREAM (Sec. 2.3) with the wall bounce-back of Sec. 3: f_k(i) <- sum_j W[k][j][i]
 * post_k(sidx[k][j][i]) for k = 0..8, then where bit k of mask[i] is set, f_k(i) <- the
 * streamed f_k'(i). */
static void orc_stream(int64_t n, int K, const int64_t *sidx, const double *W, const uint16_t *mask,
                       const double *post, double *f_out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fs[ORC_Q];
        for (int k = 0; k < ORC_Q; ++k) {
            double acc = 0.0;
            for (int j = 0; j < K; ++j) {
                int64_t t = ((int64_t)k * K + j) * n + i;
                acc += W[t] * post[(int64_t)k * n + sidx[t]];
            }
            fs[k] = acc;
        }
        for (int k = 0; k < ORC_Q; ++k) {
            double v = fs[k];
            if (mask && (mask[i] >> k & 1u)) v = fs[orc_opposite(k)];
            f_out[(int64_t)k * n + i] = v;
        }
    }
}

void orc_step(int64_t n, int K, const int64_t *sidx, const double *W, const uint16_t *mask,
              const double *gx, const double *gy, double tau, const double *f_in,
              double *f_out, double *scratch)
{
    double *post = scratch;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double f[ORC_Q], fp[ORC_Q];
        for (int k = 0; k < ORC_Q; ++k) f[k] = f_in[(int64_t)k * n + i];
        orc_collide(f, tau, gx ? gx[i] : 0.0, gy ? gy[i] : 0.0, fp);
        for (int k = 0; k < ORC_Q; ++k) post[(int64_t)k * n + i] = fp[k];
    }
    orc_stream(n, K, sidx, W, mask, post, f_out);
}

/* Collision applied to a whole field, used to express an oracle state f (post-streaming)
 * as the post-collision state f_post of the same time level. */
void orc_collide_field(int64_t n, const double *gx, const double *gy, double tau,
                       const double *f_in, double *f_out)
{
    for (int64_t i = 0; i < n; ++i) {
        double f[ORC_Q], fp[ORC_Q];
        for (int k = 0; k < ORC_Q; ++k) f[k] = f_in[(int64_t)k * n + i];
        orc_collide(f, tau, gx ? gx[i] : 0.0, gy ? gy[i] : 0.0, fp);
        for (int k = 0; k < ORC_Q; ++k) f_out[(int64_t)k * n + i] = fp[k];
    }
}

/* Moments of a whole field, eq. (macro_var). */
void orc_moments_field(int64_t n, const double *f, double *rho, double *ux, double *uy)
{
    for (int64_t i = 0; i < n; ++i) {
        double fl[ORC_Q];
        for (int k = 0; k < ORC_Q; ++k) fl[k] = f[(int64_t)k * n + i];
        orc_moments(fl, &rho[i], &ux[i], &uy[i]);
    }
}

/* Standard lattice LBM step on a periodic nx x ny lattice, node index iy*nx + ix: collide,
 * then the index-shift streaming of eq. (LBM_streaming), f_k(x) <- f_post_k(x - e_k). */
void orc_lattice_step(int nx, int ny, double tau, const double *f_in, double *f_out,
                      double *scratch)
{
    int64_t n = (int64_t)nx * ny;
    orc_collide_field(n, NULL, NULL, tau, f_in, scratch);
    for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix)
            for (int k = 0; k < ORC_Q; ++k) {
                int sx = ((ix - orc_ex[k]) % nx + nx) % nx;
                int sy = ((iy - orc_ey[k]) % ny + ny) % ny;
                f_out[(int64_t)k * n + (int64_t)iy * nx + ix] =
                    scratch[(int64_t)k * n + (int64_t)sy * nx + sx];
            }
}

/* ------------------------------------------------------------------------------------ */
/* Shan-Chen single-component multiphase extension (named in the paper's discussion as a    */
/* model whose interactions sit in the local collision; the model itself is Shan & Chen     */
/* 1993).  The paper gives no formulas: the readings are those of the library.              */
/* ------------------------------------------------------------------------------------ */

/* Pseudopotential psi(rho) = rho0 (1 - exp(-rho / rho0)). */
double orc_sc_psi(double rho, double rho0) { return rho0 * (1.0 - exp(-rho / rho0)); }

/* Interaction force at every node, F_i = -G psi_i sum_{k=1..8} omega_k psi(x_i + e_k dx_ml) e_k.
 * The point x_i + e_k dx_ml is the departure point of the opposite direction k', so psi there is
 * interpolated with the stencil and shape vector of direction k' at node i (sidx, W as in
 * orc_build_weights). */
void orc_sc_force(int64_t n, int K, const int64_t *sidx, const double *W, const double *psi, double G,
                  double *Fx, double *Fy)
{
    for (int64_t i = 0; i < n; ++i) {
        double sx = 0.0, sy = 0.0;
        for (int k = 1; k < ORC_Q; ++k) {
            int kp = orc_opposite(k);
            double pk = 0.0;
            for (int j = 0; j < K; ++j) {
                int64_t t = ((int64_t)kp * K + j) * n + i;
                pk += W[t] * psi[sidx[t]];
            }
            sx += orc_omega(k) * pk * orc_ex[k];
            sy += orc_omega(k) * pk * orc_ey[k];
        }
        Fx[i] = -G * psi[i] * sx;
        Fy[i] = -G * psi[i] * sy;
    }
}

/* Shan-Chen collision: BGK towards the equilibrium at the shifted velocity
 * u_eq = u + tau F / rho (Shan & Chen 1993), plus the body-force term of orc_collide. */
void orc_sc_collide(const double *f, double tau, double Fx, double Fy, double gx, double gy,
                    double *fpost)
{
    double rho, ux, uy;
    orc_moments(f, &rho, &ux, &uy);
    double vx = ux + tau * Fx / rho, vy = uy + tau * Fy / rho;
    for (int k = 0; k < ORC_Q; ++k) {
        double eq = orc_feq(k, rho, vx, vy);
        double force = orc_omega(k) * (orc_ex[k] * gx + orc_ey[k] * gy) / orc_cs2;
        fpost[k] = f[k] - (f[k] - eq) / tau + force;
    }
}

/* One Shan-Chen step on a cloud without walls: density of the current state at every node,
 * psi, the interaction force, the Shan-Chen collision (with the body force gx, gy if given),
 * then STREAM.  scratch holds [9][n] + 3 n doubles. */
void orc_sc_step(int64_t n, int K, const int64_t *sidx, const double *W, const double *gx,
                 const double *gy, double tau, double G, double rho0, const double *f_in,
                 double *f_out, double *scratch)
{
    double *post = scratch, *psi = scratch + (int64_t)ORC_Q * n, *Fx = psi + n, *Fy = Fx + n;
    for (int64_t i = 0; i < n; ++i) {
        double fl[ORC_Q], rho, ux, uy;
        for (int k = 0; k < ORC_Q; ++k) fl[k] = f_in[(int64_t)k * n + i];
        orc_moments(fl, &rho, &ux, &uy);
        psi[i] = orc_sc_psi(rho, rho0);
    }
    orc_sc_force(n, K, sidx, W, psi, G, Fx, Fy);
    for (int64_t i = 0; i < n; ++i) {
        double fl[ORC_Q], fp[ORC_Q];
        for (int k = 0; k < ORC_Q; ++k) fl[k] = f_in[(int64_t)k * n + i];
        orc_sc_collide(fl, tau, Fx[i], Fy[i], gx ? gx[i] : 0.0, gy ? gy[i] : 0.0, fp);
        for (int k = 0; k < ORC_Q; ++k) post[(int64_t)k * n + i] = fp[k];
    }
    orc_stream(n, K, sidx, W, NULL, post, f_out);
}

/* The Shan-Chen collision of a whole field (psi, interaction force, shifted-equilibrium BGK;
 * no streaming): the post-collision state of the same time level, as orc_collide_field.
 * scratch holds 3 n doubles. */
void orc_sc_collide_field(int64_t n, int K, const int64_t *sidx, const double *W, double tau,
                          double G, double rho0, const double *f_in, double *f_out, double *scratch)
{
    double *psi = scratch, *Fx = psi + n, *Fy = Fx + n;
    for (int64_t i = 0; i < n; ++i) {
        double fl[ORC_Q], rho, ux, uy;
        for (int k = 0; k < ORC_Q; ++k) fl[k] = f_in[(int64_t)k * n + i];
        orc_moments(fl, &rho, &ux, &uy);
        psi[i] = orc_sc_psi(rho, rho0);
    }
    orc_sc_force(n, K, sidx, W, psi, G, Fx, Fy);
    for (int64_t i = 0; i < n; ++i) {
        double fl[ORC_Q], fp[ORC_Q];
        for (int k = 0; k < ORC_Q; ++k) fl[k] = f_in[(int64_t)k * n + i];
        orc_sc_collide(fl, tau, Fx[i], Fy[i], 0.0, 0.0, fp);
        for (int k = 0; k < ORC_Q; ++k) f_out[(int64_t)k * n + i] = fp[k];
    }
}

/* The same step on a periodic nx x ny lattice with index shifts: psi(x + e_k) is the value at
 * the neighbouring lattice node, streaming as orc_lattice_step.  scratch holds [9][n] + 3 n. */
void orc_sc_lattice_step(int nx, int ny, double tau, double G, double rho0, const double *f_in,
                         double *f_out, double *scratch)
{
    int64_t n = (int64_t)nx * ny;
    double *post = scratch, *psi = scratch + (int64_t)ORC_Q * n;
    for (int64_t i = 0; i < n; ++i) {
        double fl[ORC_Q], rho, ux, uy;
        for (int k = 0; k < ORC_Q; ++k) fl[k] = f_in[(int64_t)k * n + i];
        orc_moments(fl, &rho, &ux, &uy);
        psi[i] = orc_sc_psi(rho, rho0);
    }
    for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix) {
            double sx = 0.0, sy = 0.0;
            for (int k = 1; k < ORC_Q; ++k) {
                int jx = ((ix + orc_ex[k]) % nx + nx) % nx;
                int jy = ((iy + orc_ey[k]) % ny + ny) % ny;
                double pk = psi[(int64_t)jy * nx + jx];
                sx += orc_omega(k) * pk * orc_ex[k];
                sy += orc_omega(k) * pk * orc_ey[k];
            }
            int64_t i = (int64_t)iy * nx + ix;
            double fl[ORC_Q], fp[ORC_Q];
            for (int k = 0; k < ORC_Q; ++k) fl[k] = f_in[(int64_t)k * n + i];
            orc_sc_collide(fl, tau, -G * psi[i] * sx, -G * psi[i] * sy, 0.0, 0.0, fp);
            for (int k = 0; k < ORC_Q; ++k) post[(int64_t)k * n + i] = fp[k];
        }
    for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix)
            for (int k = 0; k < ORC_Q; ++k) {
                int sxi = ((ix - orc_ex[k]) % nx + nx) % nx;
                int syi = ((iy - orc_ey[k]) % ny + ny) % ny;
                f_out[(int64_t)k * n + (int64_t)iy * nx + ix] = post[(int64_t)k * n + (int64_t)syi * nx + sxi];
            }
}

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int orc_num_threads(void) { return omp_get_max_threads(); }
void orc_set_threads(int t)
{
    if (t > 0) omp_set_num_threads(t);
}
#else
int orc_num_threads(void) { return 1; }
void orc_set_threads(int t) { (void)t; }
#endif

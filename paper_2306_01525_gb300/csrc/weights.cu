// Batched FP64 RBF-FD shape-vector solver (Sec. 2.2 eq. shape_vector, Sec. 2.3 basis r^3 + P_d,
// LU with partial pivoting) and construction of the device weights object.
//
// One warp owns one collocation system Phi_L (n = N_L + m) plus its eight right-hand sides
// (one per moving direction) as an n x (n + 8) augmented matrix in shared memory.  Lanes run
// over columns in the elimination (conflict-free row-major access) and over rows in the
// pivot search.  Systems of different sizes (batched segments) share one launch: each warp
// reads its own n from the segment table; the per-warp shared-memory slot is sized for the
// largest system of the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "mlbm_internal.h"

namespace mlbm {

__constant__ signed char c_mono_px[64];  // exponent of x of monomial l
__constant__ signed char c_mono_py[64];  // exponent of y of monomial l

namespace {

// D2Q9 directions of Sec. 2.1
__constant__ int kEx[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kEy[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

__device__ __forceinline__ double d_wrap(double d, double L) {
    if (L > 0.0) d -= L * round(d / L);
    return d;
}

__device__ __forceinline__ double d_ipow(double v, int p) {
    double r = 1.0;
    for (int i = 0; i < p; ++i) r *= v;
    return r;
}

__device__ __forceinline__ double d_mono(int l, double x, double y) {
    return d_ipow(x, c_mono_px[l]) * d_ipow(y, c_mono_py[l]);
}

constexpr int kMaxMono = (kMaxDegree + 1) * (kMaxDegree + 2) / 2;

// All monomials x^a y^b, a + b <= deg, by total degree then decreasing power of x, from
// running powers (one multiplication each).
__device__ __forceinline__ void d_monomials(int deg, double x, double y, double *out) {
    double px[kMaxDegree + 1], py[kMaxDegree + 1];
    px[0] = py[0] = 1.0;
    for (int i = 1; i <= deg; ++i) {
        px[i] = px[i - 1] * x;
        py[i] = py[i - 1] * y;
    }
    int c = 0;
    for (int t = 0; t <= deg; ++t)
        for (int b = 0; b <= t; ++b) out[c++] = px[t - b] * py[b];
}

// Cubic polyharmonic spline phi(r) = r^3 = r^2 * r.
__device__ __forceinline__ double d_phi(double dx, double dy) {
    const double r2 = dx * dx + dy * dy;
    return r2 * sqrt(r2);
}

struct SolveArgs {
    const SegDev *seg;
    const double *x, *y;
    const int32_t *idx;
    const int32_t *node_seg;
    double *w64;  // canonical [8][K][n] per segment
    unsigned long long *nbad;
    int64_t N;  // systems
    int slot;   // doubles per warp slot
    // optional system table (nearest-node stencils): system s factorises the stencil of node
    // sys_node[s] and solves for 8 evaluation points sys_q[s][c] (relative to that node,
    // physical units), writing column c to (node, direction) sys_tgt[s][c] = 8 i + k - 1 (or -1).
    // Without it system s is node s with the points -e_k dx_ml of its own 8 directions.
    const int32_t *sys_node;
    const double *sys_q;
    const int32_t *sys_tgt;
};

__device__ __forceinline__ int ld_of(int n) { return (n + 8) | 1; }

__global__ void solve_kernel(SolveArgs a) {
    extern __shared__ double sm[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double *A = sm + (size_t)warp * a.slot;
    for (int64_t sys = (int64_t)blockIdx.x * wpb + warp; sys < a.N; sys += (int64_t)gridDim.x * wpb) {
        const int64_t node = a.sys_node ? (int64_t)a.sys_node[sys] : sys;
        const SegDev sd = a.seg[a.node_seg[node]];
        const int K = sd.K, m = sd.m, n = K + m, ld = ld_of(n), nc = n + 8;
        double *tx = A + n * ld;
        double *ty = tx + K;
        double *M = ty + K;  // monomials of the scaled stencil points, [K][m]
        const int64_t il = node - sd.off;
        const double xi = a.x[node], yi = a.y[node];
        const double lx = sd.geometry == MLBM_GEOM_PERIODIC ? sd.lx : 0.0;
        const double ly = sd.geometry == MLBM_GEOM_PERIODIC ? sd.ly : 0.0;
        // stencil coordinates relative to the node (minimum image), radius
        double rmax = 0.0;
        for (int j = lane; j < K; j += 32) {
            int32_t nb = a.idx[sd.idx_off + (int64_t)j * sd.n + il];
            double dx = d_wrap(a.x[nb] - xi, lx), dy = d_wrap(a.y[nb] - yi, ly);
            tx[j] = dx;
            ty[j] = dy;
            rmax = fmax(rmax, sqrt(dx * dx + dy * dy));
        }
        for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        const double s = rmax > 0.0 ? rmax : 1.0;
        const double is = 1.0 / s;
        for (int j = lane; j < K; j += 32) {
            const double x = tx[j] * is, y = ty[j] * is;
            tx[j] = x;
            ty[j] = y;
            d_monomials(sd.deg, x, y, M + j * m);
        }
        __syncwarp();
        // augmented matrix [Phi_L | phi_L(q_1) ... phi_L(q_8)], q_k = -e_k dx_ml / s
        const double dq = sd.dx_ml * is;
        // evaluation point of right-hand side c in scaled coordinates
        auto qpt = [&](int c, double &qx, double &qy) {
            if (a.sys_node) {
                qx = a.sys_q[(sys * 8 + c) * 2] * is;
                qy = a.sys_q[(sys * 8 + c) * 2 + 1] * is;
            } else {
                qx = -kEx[c + 1] * dq;
                qy = -kEy[c + 1] * dq;
            }
        };
        // Every FP64 warp instruction costs the same whatever its active lanes (about 1.7 FP64
        // lanes per SM clock on this part, measured), so the fill, pivot search and updates are laid out
        // to keep lanes busy and keep comparisons off the FP64 unit: non-negative doubles order
        // like their bit patterns, so magnitudes are compared as 64-bit integers.
        const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
        unsigned long long amax = 0;  // bits of max |Phi entry|
        // R block: each strict upper pair evaluated once, rows a and K-2-a folded into one run of
        // K pairs; mirrored below the diagonal; phi(0) = 0 on the diagonal
        const int npair = K * (K - 1) / 2;
        for (int t = lane; t < npair; t += 32) {
            const int ra = t / K, b = t - ra * K;
            int r, c;
            if (b < K - 1 - ra) {
                r = ra;
                c = ra + 1 + b;
            } else {
                r = K - 2 - ra;
                c = b;
            }
            const double v = d_phi(tx[r] - tx[c], ty[r] - ty[c]);
            A[r * ld + c] = v;
            A[c * ld + r] = v;
            amax = max(amax, (unsigned long long)__double_as_longlong(v) & kAbs);
        }
        for (int r = lane; r < K; r += 32) A[r * ld + r] = 0.0;
        // P and P^T blocks, zero block
        for (int e = lane; e < K * m; e += 32) {
            const int r = e / m, l = e - r * m;
            const double v = M[e];
            A[r * ld + K + l] = v;
            A[(K + l) * ld + r] = v;
            amax = max(amax, (unsigned long long)__double_as_longlong(v) & kAbs);
        }
        for (int e = lane; e < m * m; e += 32) {
            const int r = e / m, l = e - r * m;
            A[(K + r) * ld + K + l] = 0.0;
        }
        // right-hand sides: phi(|q_k - x_j|) and the monomials at q_k
        for (int e = lane; e < 8 * K; e += 32) {
            const int q = e / K, r = e - q * K;
            double qx, qy;
            qpt(q, qx, qy);
            A[r * ld + n + q] = d_phi(qx - tx[r], qy - ty[r]);
        }
        if (lane < 8) {
            double qx, qy, mq[kMaxMono];
            qpt(lane, qx, qy);
            d_monomials(sd.deg, qx, qy, mq);
            for (int l = 0; l < m; ++l) A[(K + l) * ld + n + lane] = mq[l];
        }
        for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        // pivots must exceed 1e-14 max|Phi| (and be finite)
        const unsigned long long thr = (unsigned long long)__double_as_longlong(1e-14 * __longlong_as_double((long long)amax));
        __syncwarp();
        bool bad = false;
        double *invp = M + K * m;  // reciprocal pivots, [n]
        // LU with partial pivoting, eliminating the right-hand sides along
        for (int p = 0; p < n; ++p) {
            unsigned long long best = 0;
            int piv = p;
            for (int r = p + lane; r < n; r += 32) {
                const unsigned long long v = (unsigned long long)__double_as_longlong(A[r * ld + p]) & kAbs;
                if (v > best) {
                    best = v;
                    piv = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int op = __shfl_xor_sync(0xffffffffu, piv, o);
                if (ob > best || (ob == best && op < piv)) {
                    best = ob;
                    piv = op;
                }
            }
            if (!(best > thr) || best >= 0x7FF0000000000000ull) {
                bad = true;
                break;
            }
            if (piv != p) {
                for (int c = p + lane; c < nc; c += 32) {
                    double t = A[p * ld + c];
                    A[p * ld + c] = A[piv * ld + c];
                    A[piv * ld + c] = t;
                }
            }
            __syncwarp();
            const double inv = 1.0 / A[p * ld + p];
            if (lane == 0) invp[p] = inv;
            for (int r = p + 1 + lane; r < n; r += 32) A[r * ld + p] *= inv;
            __syncwarp();
            // trailing update A[r][c] -= l_r A[p][c] over the (n-p-1) x (nc-p-1) block, flattened
            // row-major across the lanes (element e = lane + 32 t), four elements per pass with
            // all loads issued before the stores
            const int C = nc - p - 1, E = (n - p - 1) * C;
            if (E > 0) {
                const int dr = 32 / C, dc = 32 - dr * C;
                int rr = lane / C, cc = lane - rr * C;
                auto advance = [&](int &r_, int &c_) {
                    r_ += dr;
                    c_ += dc;
                    if (c_ >= C) {
                        c_ -= C;
                        ++r_;
                    }
                };
                const double *Ap = A + p * ld + p + 1;   // row p, columns p+1..
                double *Ab = A + (p + 1) * ld + p + 1;   // block origin (p+1, p+1)
                const double *Al = A + (p + 1) * ld + p;  // column p, rows p+1..
                int e = lane;
                for (; e + 96 < E; e += 128) {
                    int r0 = rr, c0 = cc, r1 = r0, c1 = c0;
                    advance(r1, c1);
                    int r2 = r1, c2 = c1;
                    advance(r2, c2);
                    int r3 = r2, c3 = c2;
                    advance(r3, c3);
                    const double l0 = Al[r0 * ld], l1 = Al[r1 * ld], l2 = Al[r2 * ld], l3 = Al[r3 * ld];
                    const double u0 = Ap[c0], u1 = Ap[c1], u2 = Ap[c2], u3 = Ap[c3];
                    double a0 = Ab[r0 * ld + c0], a1 = Ab[r1 * ld + c1];
                    double a2 = Ab[r2 * ld + c2], a3 = Ab[r3 * ld + c3];
                    a0 = fma(-l0, u0, a0);
                    a1 = fma(-l1, u1, a1);
                    a2 = fma(-l2, u2, a2);
                    a3 = fma(-l3, u3, a3);
                    Ab[r0 * ld + c0] = a0;
                    Ab[r1 * ld + c1] = a1;
                    Ab[r2 * ld + c2] = a2;
                    Ab[r3 * ld + c3] = a3;
                    rr = r3;
                    cc = c3;
                    advance(rr, cc);
                }
                for (; e < E; e += 32) {
                    Ab[rr * ld + cc] = fma(-Al[rr * ld], Ap[cc], Ab[rr * ld + cc]);
                    advance(rr, cc);
                }
            }
            __syncwarp();
        }
        if (!bad) {
            // back substitution of the eight right-hand sides
            for (int p = n - 1; p >= 0; --p) {
                if (lane < 8) A[p * ld + n + lane] *= invp[p];
                __syncwarp();
                // lanes over (row, rhs) pairs; rows r = lane/8, lane/8 + 4, ... (four per pass)
                const int q = lane & 7;
                const double zq = A[p * ld + n + q];
                int r = lane >> 3;
                for (; r + 4 < p; r += 8) {
                    const double l0 = A[r * ld + p], l1 = A[(r + 4) * ld + p];
                    double a0 = A[r * ld + n + q], a1 = A[(r + 4) * ld + n + q];
                    a0 = fma(-l0, zq, a0);
                    a1 = fma(-l1, zq, a1);
                    A[r * ld + n + q] = a0;
                    A[(r + 4) * ld + n + q] = a1;
                }
                for (; r < p; r += 4) A[r * ld + n + q] = fma(-A[r * ld + p], zq, A[r * ld + n + q]);
                __syncwarp();
            }
            // polynomial reproduction check: sum_j w_j p_l(x_j) = p_l(q_k)
            double err = 0.0;
            for (int t = lane; t < 8 * m; t += 32) {
                int q = t / m, l = t - q * m;
                double acc = 0.0, qx, qy;
                qpt(q, qx, qy);
                for (int j = 0; j < K; ++j) acc = fma(A[j * ld + n + q], M[j * m + l], acc);
                err = fmax(err, fabs(acc - d_mono(l, qx, qy)));
            }
            for (int o = 16; o > 0; o >>= 1) err = fmax(err, __shfl_xor_sync(0xffffffffu, err, o));
            bad = !(err <= 1e-8);
        }
        if (bad && lane == 0) atomicAdd(a.nbad, 1ULL);
        for (int e = lane; e < 8 * K; e += 32) {
            int q = e / K, j = e - q * K;
            int64_t ti = il, tk = q;  // own mode: node il, direction q + 1
            if (a.sys_node) {
                const int32_t t = a.sys_tgt[sys * 8 + q];
                if (t < 0) continue;
                ti = (int64_t)(t >> 3) - sd.off;
                tk = t & 7;
            }
            double v = bad ? 0.0 : A[j * ld + n + q];
            a.w64[sd.w_off + (tk * K + j) * sd.n + ti] = v;
        }
        __syncwarp();
    }
}

// FP32 shape vectors that keep the polynomial reproduction of eq. (shape_vector).
//
// The FP32 step interpolates in difference form, fhat = f(c) + sum_{j>=1} w_j (f(s_j) - f(c))
// with c the stencil's centre member, so constants are reproduced exactly whatever the weights.
// Rounding each FP64 weight to the nearest float leaves sum_{j>=1} (w32_j - w_j) p(x_j) != 0
// for the monomials p of degree 1..d (taken about the centre): a fixed per-node error of the
// interpolated gradient and curvature that repeats every step, so it accumulates coherently
// over a run (5e-6 relative L2 of u after 300 steps on a 400-node cloud with N_L = 30, P_4).
// Here the weights of one (node, direction) are rounded one at a time, largest |w| first, and
// each is rounded at w_j + delta_j, where delta_j is the j-th entry of the minimum-norm
// correction of the weights not yet rounded that cancels the moment error R accumulated so far:
// delta_j = -a_j^T (G + lambda I)^{-1} R with a_j the monomial vector of member j and G the Gram
// matrix of the members not yet rounded.  The error that remains is that of the last, smallest
// weights, whose floats are finest.  R, G and the corrections are carried in FP32 in
// coordinates scaled by the stencil radius (|a_j| <= 1); only w_j + delta_j and its rounding
// are FP64.  A correction larger than 2^-12 max|w| (or a failed factorisation) is dropped,
// so a weight never moves by more than that from its FP64 value.
constexpr int kRoundMaxDeg = 6;  // moments corrected up to degree min(d, 6)
constexpr float kRoundLambda = 1e-3f;

__device__ __forceinline__ double d_wrap2(double d, double L) {
    if (L > 0.0) d -= L * round(d / L);
    return d;
}

template <int D>
__global__ void __launch_bounds__(128) round32_kernel(const SegDev *__restrict__ segs, int s,
                                                      const double *__restrict__ x, const double *__restrict__ y,
                                                      const int32_t *__restrict__ idx,
                                                      const int32_t *__restrict__ near,
                                                      const double *__restrict__ w64c, float *__restrict__ w32c) {
    constexpr int M = (D + 1) * (D + 2) / 2 - 1;  // monomials of degree 1..D
    constexpr int P = M * (M + 1) / 2;            // packed lower triangle
    const SegDev sd = segs[s];
    const int K = sd.K, nw = K - 1;
    const int64_t n = sd.n;
    const double lx = sd.geometry == MLBM_GEOM_PERIODIC ? sd.lx : 0.0;
    const double ly = sd.geometry == MLBM_GEOM_PERIODIC ? sd.ly : 0.0;
    float px[kMaxK], py[kMaxK];
    double wv[kMaxK];
    unsigned char ord[kMaxK];
    float G[P], Lc[P], Li[M], R[M], a[M], v[M];
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < 8 * n; g += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(g / n);  // direction k + 1
        const int64_t i = g - (int64_t)k * n;
        // stencil that interpolates (i, k + 1): the node's own, or its departure node's
        const int64_t L = near ? (int64_t)near[8 * sd.off + (int64_t)k * n + i] - sd.off : i;
        const int32_t c = idx[sd.idx_off + L];
        const double xc = x[c], yc = y[c];
        double rmax = 0.0, wmax = 0.0;
        const double *wk = w64c + sd.w_off + (int64_t)k * K * n + i;
        for (int j = 0; j < nw; ++j) {
            const int32_t m = idx[sd.idx_off + (int64_t)(j + 1) * n + L];
            const double dx = d_wrap2(x[m] - xc, lx), dy = d_wrap2(y[m] - yc, ly);
            rmax = fmax(rmax, sqrt(dx * dx + dy * dy));
            px[j] = (float)dx;
            py[j] = (float)dy;
            wv[j] = wk[(int64_t)(j + 1) * n];
            wmax = fmax(wmax, fabs(wv[j]));
        }
        const float is = rmax > 0.0 ? (float)(1.0 / rmax) : 1.f;
        // order: largest |w| first (stable)
        for (int j = 0; j < nw; ++j) {
            int t = j;
            const double aj = fabs(wv[j]);
            while (t > 0 && fabs(wv[ord[t - 1]]) < aj) {
                ord[t] = ord[t - 1];
                --t;
            }
            ord[t] = (unsigned char)j;
        }
        auto mono = [&](int j, float (&out)[M]) {
            const float u = px[j] * is, w = py[j] * is;
            float pu[D + 1], pw[D + 1];
            pu[0] = pw[0] = 1.f;
#pragma unroll
            for (int t = 1; t <= D; ++t) {
                pu[t] = pu[t - 1] * u;
                pw[t] = pw[t - 1] * w;
            }
            int q = 0;
#pragma unroll
            for (int t = 1; t <= D; ++t)
#pragma unroll
                for (int b = 0; b <= t; ++b) out[q++] = pu[t - b] * pw[b];
        };
#pragma unroll
        for (int e = 0; e < P; ++e) G[e] = 0.f;
#pragma unroll
        for (int r = 0; r < M; ++r) R[r] = 0.f;
        for (int j = 0; j < nw; ++j) {
            mono(j, a);
#pragma unroll
            for (int r = 0, e = 0; r < M; ++r)
#pragma unroll
                for (int q = 0; q <= r; ++q, ++e) G[e] = fmaf(a[r], a[q], G[e]);
        }
        const double bound = wmax * 0x1p-12;
        float *out = w32c + sd.w_off + (int64_t)k * K * n + i;
        out[0] = (float)wk[0];  // centre: not read by the FP32 difference form
        bool ok = true;
        for (int p = 0; p < nw; ++p) {
            const int j = ord[p];
            mono(j, a);
            // Cholesky of G + lambda I (refactorised every second entry: the factor of the Gram
            // matrix that still holds the previous entry serves the next one), then
            // v = (G + lambda I)^{-1} R; the diagonal is kept as reciprocals
            if ((p & 1) == 0) {
                ok = true;
                for (int r = 0, er = 0; r < M; er += ++r) {
                    for (int q = 0; q <= r; ++q) {
                        const int eq = q * (q + 1) / 2;
                        float t = G[er + q] + (q == r ? kRoundLambda : 0.f);
                        for (int u = 0; u < q; ++u) t = fmaf(-Lc[er + u], Lc[eq + u], t);
                        if (q == r) {
                            ok = ok && t > 0.f;
                            Li[r] = t > 0.f ? 1.f / sqrtf(t) : 1.f;
                            Lc[er + r] = 1.f;
                        } else {
                            Lc[er + q] = t * Li[q];
                        }
                    }
                }
            }
            double delta = 0.0;
            if (ok) {
                for (int r = 0, er = 0; r < M; er += ++r) {
                    float t = R[r];
                    for (int q = 0; q < r; ++q) t = fmaf(-Lc[er + q], v[q], t);
                    v[r] = t * Li[r];
                }
                for (int r = M - 1; r >= 0; --r) {
                    float t = v[r];
                    for (int q = r + 1; q < M; ++q) t = fmaf(-Lc[q * (q + 1) / 2 + r], v[q], t);
                    v[r] = t * Li[r];
                }
                float dot = 0.f;
#pragma unroll
                for (int r = 0; r < M; ++r) dot = fmaf(a[r], v[r], dot);
                delta = -(double)dot;
                if (!(fabs(delta) <= bound)) delta = 0.0;
            }
            const float w32 = __double2float_rn(wv[j] + delta);
            const float rho = (float)((double)w32 - wv[j]);
#pragma unroll
            for (int r = 0, e = 0; r < M; ++r) {
                R[r] = fmaf(rho, a[r], R[r]);
#pragma unroll
                for (int q = 0; q <= r; ++q, ++e) G[e] = fmaf(-a[r], a[q], G[e]);
            }
            out[(int64_t)(j + 1) * n] = w32;
        }
    }
}

// Canonical [8][K][n] shape vectors -> tile layouts of the fused step:
//   FP32 (members j = 1..K-1, from the rounded canonical FP32 array):
//        element (((j-1) * 2 + h) * B + b) * 4 + r, k = 1 + 4 h + r
//   FP64 (members j = 0..K-1): element ((j * 4 + q) * B + b) * 2 + r,     k = 1 + 2 q + r
// with B the tile size of the weights object.
__global__ void repack_kernel(const TileDev *__restrict__ tiles, int ntiles, const SegDev *__restrict__ seg,
                              const double *__restrict__ w64c, const float *__restrict__ w32c,
                              float *__restrict__ w32t, double *__restrict__ w64t, int B) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileDev tile = tiles[t];
        const SegDev &sd = seg[tile.seg];
        const int K = tile.K;
        const int64_t il0 = tile.begin - sd.off;
        if (w32t) {
            const int64_t total = (int64_t)(K - 1) * 8 * B;
            for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
                const int r = (int)(e & 3);
                const int64_t q4 = e >> 2;
                const int b = (int)(q4 % B);
                const int64_t jh = q4 / B;
                const int h = (int)(jh & 1), j = (int)(jh >> 1) + 1, k = 1 + 4 * h + r;
                w32t[tile.w_off + e] = b < tile.count ? w32c[sd.w_off + ((int64_t)(k - 1) * K + j) * sd.n + il0 + b] : 0.f;
            }
        }
        if (w64t) {
            const int64_t total = (int64_t)K * 8 * B;
            for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
                const int r = (int)(e & 1);
                const int64_t q2 = e >> 1;
                const int b = (int)(q2 % B);
                const int64_t jq = q2 / B;
                const int q = (int)(jq & 3), j = (int)(jq >> 2), k = 1 + 2 * q + r;
                double v = b < tile.count ? w64c[sd.w_off + ((int64_t)(k - 1) * K + j) * sd.n + il0 + b] : 0.0;
                w64t[tile.w64_off + e] = v;
            }
        }
    }
}

template <typename T>
int dev_alloc(T **p, size_t count, const char *what) {
    *p = nullptr;
    if (count == 0) return MLBM_OK;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? MLBM_ENOMEM : MLBM_ECUDA,
                    std::string("cudaMalloc failed for ") + what + ": " + cudaGetErrorString(e));
    }
    return MLBM_OK;
}

int cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MLBM_OK;
    return fail(MLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void free_weights(mlbm_weights *w) {
    if (!w) return;
    for (auto &kv : w->graphs) cudaGraphExecDestroy((cudaGraphExec_t)kv.second);
    w->graphs.clear();
    cudaFree(w->d_seg);
    cudaFree(w->d_tiles);
    cudaFree(w->d_idx);
    cudaFree(w->d_w64);
    cudaFree(w->d_w32t);
    cudaFree(w->d_w32c);
    cudaFree(w->d_x);
    cudaFree(w->d_y);
    cudaFree(w->d_w64t);
    cudaFree(w->d_lidx);
    cudaFree(w->d_halo);
    cudaFree(w->d_mask);
    cudaFree(w->d_fdir32);
    cudaFree(w->d_fdir64);
    cudaFree(w->d_perm);
    cudaFree(w->d_node_seg);
    cudaFree(w->d_csr_ptr);
    cudaFree(w->d_csr_ent);
    cudaFree(w->d_scratch);
    cudaFree(w->d_partials);
    cudaFree(w->d_params);
    cudaFree(w->d_sc);
    cudaFree(w->d_sc_psi);
    cudaFree(w->d_tiles_run);
    cudaFree(w->d_adj_rowp);
    cudaFree(w->d_adj_rhalo);
    cudaFree(w->d_adj_roff);
    cudaFree(w->d_adj_rcnt);
    cudaFree(w->d_adj_sbeg);
    cudaFree(w->d_adj_cbeg);
    cudaFree(w->d_adj_slen);
    cudaFree(w->d_adj_nlen);
    cudaFree(w->d_adj_slot);
    cudaFree(w->d_adj_src);
    cudaFree(w->d_adj_jh);
    cudaFree(w->d_near);
    for (void *b : w->d_adj_coef) cudaFree(b);
    for (void *b : w->d_stage) cudaFree(b);
    for (void *q : w->copy_stream)
        if (q) cudaStreamDestroy((cudaStream_t)q);
    for (void *e : w->stage_event)
        if (e) cudaEventDestroy((cudaEvent_t)e);
    delete w;
}

}  // namespace

// Solve all systems of a weights object (device arrays must be in place).  Returns the number
// of bad systems through nbad_out.
struct SolveShape {
    int slot;    // doubles per warp
    int nmax;
};

static SolveShape solve_shape(const mlbm_weights *w) {
    int nmax = 0, kmax = 0;
    for (auto &s : w->seg) {
        nmax = std::max(nmax, s.K + s.m);
        kmax = std::max(kmax, s.K);
    }
    int km = 0;
    for (auto &s : w->seg) km = std::max(km, s.K * s.m);
    const int ld = (nmax + 8) | 1;
    return SolveShape{nmax * ld + 2 * kmax + km + nmax, nmax};
}

// Launch the solver over nodes [0, count) with `wpb` warps (one system each) per CTA.
static int launch_solve(mlbm_weights *w, const double *d_x, const double *d_y, unsigned long long *d_bad,
                        int64_t count, int wpb, cudaStream_t st) {
    const SolveShape sh = solve_shape(w);
    const size_t smem = (size_t)wpb * sh.slot * sizeof(double);
    int rc = allow_dynamic_smem((const void *)solve_kernel);
    if (rc) return rc;
    SolveArgs a;
    a.seg = w->d_seg;
    a.x = d_x;
    a.y = d_y;
    a.idx = w->d_idx;
    a.node_seg = w->d_node_seg;
    a.w64 = w->d_w64;
    a.nbad = d_bad;
    a.N = count;
    a.slot = sh.slot;
    a.sys_node = w->d_sys_node;
    a.sys_q = w->d_sys_q;
    a.sys_tgt = w->d_sys_tgt;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel, 32 * wpb, smem);
    const int64_t need = (count + wpb - 1) / wpb;
    const int64_t grid = std::min<int64_t>(need, (int64_t)std::max(1, per_sm) * w->num_sms);
    solve_kernel<<<(unsigned)grid, 32 * wpb, smem, st>>>(a);
    return cuda_check(cudaGetLastError(), "solve_kernel launch");
}

// Autotuner of the batched solver's CTA shape: for launches of at least `kTuneMin` systems,
// each warps-per-CTA candidate that fits in shared memory is timed (CUDA events) on the first
// systems of the batch and the fastest is kept, cached per largest system size.
static int tune_warps(mlbm_weights *w, const double *d_x, const double *d_y, unsigned long long *d_bad,
                      cudaStream_t st, int *best_wpb) {
    static std::map<int, int> cache;
    static std::mutex cache_mu;
    const SolveShape sh = solve_shape(w);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, w->device);
    auto fits = [&](int wpb) { return (size_t)wpb * sh.slot * sizeof(double) <= (size_t)maxsm; };
    *best_wpb = 0;
    for (int wpb = 4; wpb >= 1; wpb >>= 1)
        if (fits(wpb)) {
            *best_wpb = wpb;
            break;
        }
    if (!*best_wpb) return fail(MLBM_EINVAL, "collocation system too large for shared memory");
    constexpr int64_t kTuneMin = 200000;
    const int64_t nsys = w->d_sys_node ? w->nsys : w->N;
    if (nsys < kTuneMin) return MLBM_OK;
    {
        std::lock_guard<std::mutex> lk(cache_mu);
        auto it = cache.find(sh.nmax);
        if (it != cache.end() && fits(it->second)) {
            *best_wpb = it->second;
            return MLBM_OK;
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    const int64_t sample = std::min<int64_t>(nsys, (int64_t)w->num_sms * 96);
    for (int wpb : {1, 2, 4, 8, 12, 16}) {
        if (!fits(wpb)) continue;
        int rc = launch_solve(w, d_x, d_y, d_bad, sample, wpb, st);  // warm the configuration
        if (!rc) {
            cudaEventRecord(e0, st);
            rc = launch_solve(w, d_x, d_y, d_bad, sample, wpb, st);
            cudaEventRecord(e1, st);
        }
        if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "solver tuning");
        if (rc) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            *best_wpb = wpb;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(cache_mu);
    cache[sh.nmax] = *best_wpb;
    return MLBM_OK;
}

// System table of a cloud with nearest-node stencils: every departure point x_i - e_k dx_ml
// is assigned to the node L whose stencil interpolates it; the points of each L are solved
// against L's factorised collocation matrix in groups of up to eight right-hand sides.
static void build_systems(const mlbm_cloud *c, std::vector<int32_t> &node, std::vector<double> &q,
                          std::vector<int32_t> &tgt) {
    static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    node.clear();
    q.clear();
    tgt.clear();
    auto wrap = [](double d, double L) { return L > 0.0 ? d - L * std::round(d / L) : d; };
    for (int s = 0; s < c->nseg; ++s) {
        const SegmentHost &h = c->seg[s];
        const double lx = h.d.geometry == MLBM_GEOM_PERIODIC ? h.d.lx : 0.0;
        const double ly = h.d.geometry == MLBM_GEOM_PERIODIC ? h.d.ly : 0.0;
        const int32_t *near = &c->near[(size_t)8 * h.off];
        // pairs (i, k) grouped by their departure node L (counting sort, i then k ascending)
        std::vector<int64_t> start(h.n + 1, 0);
        for (int k = 0; k < 8; ++k)
            for (int64_t i = 0; i < h.n; ++i) start[near[(int64_t)k * h.n + i] - h.off + 1]++;
        for (int64_t L = 0; L < h.n; ++L) start[L + 1] += start[L];
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        std::vector<int32_t> pairs((size_t)8 * h.n);
        for (int64_t i = 0; i < h.n; ++i)
            for (int k = 0; k < 8; ++k) {
                const int64_t L = near[(int64_t)k * h.n + i] - h.off;
                pairs[fill[L]++] = (int32_t)(i * 8 + k);
            }
        for (int64_t L = 0; L < h.n; ++L)
            for (int64_t b = start[L]; b < start[L + 1]; b += 8) {
                node.push_back((int32_t)(h.off + L));
                for (int c8 = 0; c8 < 8; ++c8) {
                    if (b + c8 < start[L + 1]) {
                        const int32_t pr = pairs[b + c8];
                        const int64_t i = pr >> 3;
                        const int k = (pr & 7) + 1;
                        const double Dx = c->x[h.off + i] - ex[k] * h.d.dx_ml;
                        const double Dy = c->y[h.off + i] - ey[k] * h.d.dx_ml;
                        q.push_back(wrap(Dx - c->x[h.off + L], lx));
                        q.push_back(wrap(Dy - c->y[h.off + L], ly));
                        tgt.push_back((int32_t)((h.off + i) * 8 + (k - 1)));
                    } else {
                        q.push_back(0.0);
                        q.push_back(0.0);
                        tgt.push_back(-1);
                    }
                }
            }
    }
}

// Solve all systems of a weights object (device arrays in place).  warps_per_block <= 0 asks
// the autotuner.  The number of bad systems is returned through nbad_out.
int solve_weights(mlbm_weights *w, const double *d_x, const double *d_y, cudaStream_t st,
                  int warps_per_block, int64_t *nbad_out) {
    unsigned long long *d_bad = nullptr;
    int rc = dev_alloc(&d_bad, 1, "bad counter");
    if (rc) return rc;
    int wpb = warps_per_block;
    if (wpb <= 0) rc = tune_warps(w, d_x, d_y, d_bad, st, &wpb);
    if (!rc) rc = cuda_check(cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), st), "memset");
    if (!rc) rc = launch_solve(w, d_x, d_y, d_bad, w->d_sys_node ? w->nsys : w->N, wpb, st);
    unsigned long long nbad = 0;
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&nbad, d_bad, sizeof(nbad), cudaMemcpyDeviceToHost, st), "copy");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "solve_kernel");
    cudaFree(d_bad);
    w->solve_wpb = wpb;
    if (nbad_out) *nbad_out = (int64_t)nbad;
    return rc;
}

// Rounded canonical FP32 shape vectors of every segment (round32_kernel at the segment's
// degree, at most kRoundMaxDeg).
int round_weights32(mlbm_weights *w, cudaStream_t st) {
    int rc = MLBM_OK;
    for (int s = 0; s < w->nseg && !rc; ++s) {
        const SegmentHost &h = w->seg[s];
        if (h.n == 0) continue;
        const int D = std::max(1, std::min(kRoundMaxDeg, h.d.degree));
        const int64_t total = 8 * h.n;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 127) / 128, 32 * (int64_t)w->num_sms));
        const int32_t *near = h.d.stencil_mode == MLBM_STENCIL_NEAREST ? w->d_near : nullptr;
        if (h.d.stencil_mode == MLBM_STENCIL_NEAREST && !near) return fail(MLBM_EINVAL, "departure nodes missing");
#define MLBM_ROUND32(DD)                                                                                         \
    case DD:                                                                                                     \
        round32_kernel<DD><<<grid, 128, 0, st>>>(w->d_seg, s, w->d_x, w->d_y, w->d_idx, near, w->d_w64, w->d_w32c); \
        break;
        switch (D) {
            MLBM_ROUND32(1)
            MLBM_ROUND32(2)
            MLBM_ROUND32(3)
            MLBM_ROUND32(4)
            MLBM_ROUND32(5)
            MLBM_ROUND32(6)
        }
#undef MLBM_ROUND32
        rc = cuda_check(cudaGetLastError(), "FP32 rounding launch");
    }
    return rc;
}

// Refresh the tile layouts from the canonical FP64 shape vectors.
int repack_weights(mlbm_weights *w, cudaStream_t st) {
    if (!w->d_w32t && !w->d_w64t) return MLBM_OK;
    int rc = w->d_w32t ? round_weights32(w, st) : MLBM_OK;
    if (rc) return rc;
    int grid = std::max(1, std::min(w->ntiles, 8 * w->num_sms));
    repack_kernel<<<grid, 256, 0, st>>>(w->d_tiles, w->ntiles, w->d_seg, w->d_w64, w->d_w32c, w->d_w32t,
                                        w->d_w64t, w->tile_nodes);
    rc = cuda_check(cudaGetLastError(), "repack launch");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "repack");
    return rc;
}

int build_tiles(const mlbm_cloud *c, int B, std::vector<TileDev> &tiles, std::vector<int32_t> &halo,
                std::vector<uint32_t> &lidx, int &umax, int64_t &wt_total, int64_t &wt64_total);

}  // namespace mlbm

using namespace mlbm;

namespace {

int upload_monomial_tables() {
    signed char px[64] = {0}, py[64] = {0};
    int c = 0;
    for (int t = 0; t <= kMaxDegree; ++t)
        for (int b = 0; b <= t; ++b) {
            px[c] = (signed char)(t - b);
            py[c] = (signed char)b;
            ++c;
        }
    cudaError_t e = cudaMemcpyToSymbol(c_mono_px, px, sizeof(px));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_mono_py, py, sizeof(py));
    return e == cudaSuccess ? MLBM_OK : fail(MLBM_ECUDA, std::string("monomial tables: ") + cudaGetErrorString(e));
}

template <typename T>
int upload(T **dst, const T *src, size_t count, const char *what) {
    int rc = dev_alloc(dst, count, what);
    if (rc) return rc;
    if (count == 0) return MLBM_OK;
    return cuda_check(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice), what);
}

}  // namespace

namespace mlbm {
int prepare_step_grids(mlbm_weights *w);
}

extern "C" {

int mlbm_build_weights(const mlbm_cloud *c, int flags, void *stream, mlbm_weights **out,
                       int64_t *n_bad) {
    set_error("");
    if (!c || !out) return fail(MLBM_EINVAL, "NULL argument");
    *out = nullptr;
    if (flags == 0) flags = MLBM_KEEP_W32 | MLBM_KEEP_W64;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(MLBM_ECUDA, "no usable CUDA device");
    }
    cudaStream_t st = (cudaStream_t)stream;
    mlbm_weights *w = new (std::nothrow) mlbm_weights();
    if (!w) return fail(MLBM_ENOMEM, "host allocation failed");
    w->device = dev;
    cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev);
    w->nseg = c->nseg;
    w->N = c->N;
    w->seg = c->seg;
    w->perm = c->perm;
    w->idx_total = c->idx_total;
    w->w_total = c->w_total;
    {
        std::vector<int64_t> ns;
        for (auto &h : c->seg) ns.push_back(h.n);
        w->tile_nodes = choose_tile_nodes(ns, w->num_sms);
    }
    int rc = upload_monomial_tables();
    // segment table
    std::vector<SegDev> sd(c->nseg);
    for (int s = 0; s < c->nseg; ++s) {
        const SegmentHost &h = c->seg[s];
        sd[s].off = h.off;
        sd[s].n = h.n;
        sd[s].idx_off = h.idx_off;
        sd[s].w_off = h.w_off;
        sd[s].K = h.K;
        sd[s].m = h.m;
        sd[s].deg = h.d.degree;
        sd[s].geometry = h.d.geometry;
        sd[s].lx = h.d.lx;
        sd[s].ly = h.d.ly;
        sd[s].dx_ml = h.d.dx_ml;
        sd[s].pad = 0;
    }
    // tiles of the fused step with their halos and packed stencil slots
    std::vector<TileDev> tiles;
    std::vector<int32_t> halo;
    std::vector<uint32_t> lidx;
    if (!rc) rc = build_tiles(c, w->tile_nodes, tiles, halo, lidx, w->umax, w->wt_total, w->wt64_total);
    if (rc) {
        free_weights(w);
        return rc;
    }
    w->l_total = (int64_t)lidx.size();
    w->h_total = (int64_t)halo.size();
    w->ntiles = (int)tiles.size();
    bool any_mask = false;
    for (auto m : c->mask) any_mask |= (m != 0);
    w->has_mask = any_mask;
    std::vector<float> fd32(c->fdir.begin(), c->fdir.end());
    if (!rc) rc = upload(&w->d_seg, sd.data(), sd.size(), "segments");
    if (!rc) rc = upload(&w->d_tiles, tiles.data(), tiles.size(), "tiles");
    if (!rc) rc = upload(&w->d_idx, c->idx.data(), c->idx.size(), "stencil");
    if (!rc) rc = upload(&w->d_mask, c->mask.data(), c->mask.size(), "mask");
    if (!rc) rc = upload(&w->d_fdir64, c->fdir.data(), c->fdir.size(), "force direction");
    if (!rc) rc = upload(&w->d_fdir32, fd32.data(), fd32.size(), "force direction");
    if (!rc) rc = upload(&w->d_perm, c->perm.data(), c->perm.size(), "permutation");
    if (!rc) rc = upload(&w->d_node_seg, c->node_seg.data(), c->node_seg.size(), "node segments");
    if (!rc) rc = upload(&w->d_csr_ptr, c->csr_ptr.data(), c->csr_ptr.size(), "transposed stencil");
    if (!rc) rc = upload(&w->d_csr_ent, c->csr_ent.data(), c->csr_ent.size(), "transposed stencil");
    if (!rc) rc = upload(&w->d_x, c->x.data(), c->x.size(), "x");
    if (!rc) rc = upload(&w->d_y, c->y.data(), c->y.size(), "y");
    if (!rc) rc = upload(&w->d_halo, halo.data(), halo.size(), "halo lists");
    if (!rc) rc = upload(&w->d_lidx, lidx.data(), lidx.size(), "stencil slots");
    if (!rc) rc = dev_alloc(&w->d_w64, (size_t)w->w_total, "W64");
    if (!rc && (flags & MLBM_KEEP_W64)) rc = dev_alloc(&w->d_w64t, (size_t)w->wt64_total, "W64 tiles");
    if (!rc && (flags & MLBM_KEEP_W32)) rc = dev_alloc(&w->d_w32t, (size_t)w->wt_total, "W32 tiles");
    if (!rc && (flags & MLBM_KEEP_W32)) rc = dev_alloc(&w->d_w32c, (size_t)w->w_total, "W32");
    if (!rc) rc = dev_alloc(&w->d_params, (size_t)6 * c->nseg, "params");
    int64_t nbad = 0;
    for (auto &h : c->seg) w->any_nearest |= h.d.stencil_mode == MLBM_STENCIL_NEAREST;
    if (!rc && w->any_nearest) {
        std::vector<int32_t> sn, stg;
        std::vector<double> sq;
        build_systems(c, sn, sq, stg);
        w->nsys = (int64_t)sn.size();
        rc = upload(&w->d_sys_node, sn.data(), sn.size(), "system table");
        if (!rc) rc = upload(&w->d_sys_q, sq.data(), sq.size(), "system table");
        if (!rc) rc = upload(&w->d_sys_tgt, stg.data(), stg.size(), "system table");
        // departure nodes, kept for the adjoint's transposed interpolation
        if (!rc) rc = upload(&w->d_near, c->near.data(), c->near.size(), "departure nodes");
    }
    if (!rc) rc = solve_weights(w, w->d_x, w->d_y, st, 0, &nbad);
    cudaFree(w->d_sys_node);
    cudaFree(w->d_sys_q);
    cudaFree(w->d_sys_tgt);
    w->d_sys_node = w->d_sys_tgt = nullptr;
    w->d_sys_q = nullptr;
    if (!rc) rc = repack_weights(w, st);
    if (rc) {
        free_weights(w);
        return rc;
    }
    if ((rc = prepare_step_grids(w))) {
        free_weights(w);
        return rc;
    }
    if (n_bad) *n_bad = nbad;
    *out = w;
    if (nbad > 0)
        return fail(MLBM_ESINGULAR, std::to_string(nbad) + " collocation systems singular or inaccurate");
    return MLBM_OK;
}

void mlbm_weights_free(mlbm_weights *w) { free_weights(w); }

int mlbm_weights_info(const mlbm_weights *w, int64_t *n_nodes, int *nseg) {
    if (!w) return fail(MLBM_EINVAL, "NULL weights");
    if (n_nodes) *n_nodes = w->N;
    if (nseg) *nseg = w->nseg;
    return MLBM_OK;
}

int mlbm_weights_download(const mlbm_weights *w, int seg, double *W) {
    if (!w || !W) return fail(MLBM_EINVAL, "NULL argument");
    if (seg < 0 || seg >= w->nseg) return fail(MLBM_EINVAL, "segment out of range");
    const SegmentHost &h = w->seg[seg];
    size_t cnt = (size_t)8 * h.K * h.n;
    std::vector<double> tmp(cnt);
    int rc = cuda_check(cudaMemcpy(tmp.data(), w->d_w64 + h.w_off, cnt * sizeof(double), cudaMemcpyDeviceToHost),
                        "download weights");
    if (rc) return rc;
    for (int64_t p = 0; p < h.n; ++p) {
        int64_t io = w->perm[h.off + p] - h.orig_off;
        for (int64_t r = 0; r < (int64_t)8 * h.K; ++r) W[r * h.n + io] = tmp[r * h.n + p];
    }
    return MLBM_OK;
}

int mlbm_weights_download_f32(const mlbm_weights *w, int seg, float *W) {
    if (!w || !W) return fail(MLBM_EINVAL, "NULL argument");
    if (seg < 0 || seg >= w->nseg) return fail(MLBM_EINVAL, "segment out of range");
    if (!w->d_w32c) return fail(MLBM_EINVAL, "weights built without MLBM_KEEP_W32");
    const SegmentHost &h = w->seg[seg];
    size_t cnt = (size_t)8 * h.K * h.n;
    std::vector<float> tmp(cnt);
    int rc = cuda_check(cudaMemcpy(tmp.data(), w->d_w32c + h.w_off, cnt * sizeof(float), cudaMemcpyDeviceToHost),
                        "download FP32 weights");
    if (rc) return rc;
    for (int64_t p = 0; p < h.n; ++p) {
        int64_t io = w->perm[h.off + p] - h.orig_off;
        for (int64_t r = 0; r < (int64_t)8 * h.K; ++r) W[r * h.n + io] = tmp[r * h.n + p];
    }
    return MLBM_OK;
}

int mlbm_weights_upload(mlbm_weights *w, int seg, const double *W, const int32_t *idx) {
    if (!w || !W || !idx) return fail(MLBM_EINVAL, "NULL argument");
    if (seg < 0 || seg >= w->nseg) return fail(MLBM_EINVAL, "segment out of range");
    const SegmentHost &h = w->seg[seg];
    // check the caller's stencil against ours (original numbering)
    std::vector<int32_t> own((size_t)h.K * h.n);
    int rc = cuda_check(cudaMemcpy(own.data(), w->d_idx + h.idx_off, own.size() * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost),
                        "download stencil");
    if (rc) return rc;
    for (int j = 0; j < h.K; ++j)
        for (int64_t p = 0; p < h.n; ++p) {
            int64_t io = w->perm[h.off + p] - h.orig_off;
            int64_t member = w->perm[own[(size_t)j * h.n + p]] - h.orig_off;
            if (idx[(int64_t)j * h.n + io] != member)
                return fail(MLBM_EINVAL, "stencil differs from the library's stencil");
        }
    size_t cnt = (size_t)8 * h.K * h.n;
    std::vector<double> tmp(cnt);
    for (int64_t p = 0; p < h.n; ++p) {
        int64_t io = w->perm[h.off + p] - h.orig_off;
        for (int64_t r = 0; r < (int64_t)8 * h.K; ++r) tmp[r * h.n + p] = W[r * h.n + io];
    }
    if ((rc = cuda_check(cudaMemcpy(w->d_w64 + h.w_off, tmp.data(), cnt * sizeof(double), cudaMemcpyHostToDevice),
                         "upload weights")))
        return rc;
    if ((rc = repack_weights(w, nullptr))) return rc;
    // the adjoint's transposed coefficients hold the old shape vectors: drop them, so the next
    // reverse step rebuilds them (its slot tables depend on the stencils only, checked above)
    if (w->d_adj_coef[0] || w->d_adj_coef[1]) {
        if ((rc = cuda_check(cudaDeviceSynchronize(), "upload weights"))) return rc;
        for (void *&c : w->d_adj_coef) {
            cudaFree(c);
            c = nullptr;
        }
    }
    return MLBM_OK;
}

}  // extern "C"

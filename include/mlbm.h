/*
 * mlbm.h -- C ABI of the GB300 meshless lattice Boltzmann library.
 *
 * The method is the semi-Lagrangian meshless LBM of Strzelczyk & Matyka (arXiv 2306.01525):
 * D2Q9 BGK populations live on a scattered node cloud; every time step interpolates the
 * post-collision populations at the departure points x_i - e_k dx_ml with RBF-FD shape
 * vectors (cubic polyharmonic spline r^3 plus polynomials of total degree <= d) precomputed
 * once over each node's N_L-nearest-neighbour stencil, then collides locally.
 *
 * Conventions (all entry points):
 *  - Every function returns an int status (MLBM_OK or a negative MLBM_E* code) unless noted;
 *    mlbm_last_error() returns a thread-local message for the last failure on that thread.
 *  - Sizes and counts are int64_t.  Host pointers are read during the call only.
 *  - Opaque objects (mlbm_cloud, mlbm_weights) are created and freed by the library.
 *  - Field buffers are owned by the caller.  "device" pointers must be CUDA device memory of
 *    the current device; "host" pointers are ordinary host memory.
 *  - Work taking a `stream` argument (a cudaStream_t passed as void*, NULL = legacy default
 *    stream) is enqueued asynchronously on that stream; errors raised by kernels surface at
 *    the next call that synchronises.  Nothing here falls back to the CPU: without a usable
 *    CUDA device every GPU entry point fails with MLBM_ECUDA.
 *  - A weights object keeps one device copy of the step parameters (and of the Shan-Chen
 *    couplings), refreshed on the calling stream when they change.  All calls that use one
 *    weights object must therefore be ordered with one another: issue them on one stream (or
 *    order the streams with events).  Two calls with different parameters on two unordered
 *    streams race: the earlier call's kernels may read the later call's parameters.  Calls on
 *    one weights object must not run concurrently from several host threads either.
 *  - Node order: the library stores nodes in Morton (Z-curve) order within each segment;
 *    "stored order" below means that order, "original order" the caller's input order.
 *    mlbm_cloud_perm gives the mapping.
 *  - State layout: populations are SoA, f[k * N + p] for k = 0..8 and stored position p,
 *    N the total node count.  dtype MLBM_F64 stores the populations themselves;
 *    dtype MLBM_F32 stores deviations f_k - omega_k * rho0 (rho0 from mlbm_params).
 *    The state held between steps is the post-collision population f^post (Sec. 2.1,
 *    eq. LBM_collision), so that one step is pull-stream, bounce-back, collide.
 *  - D2Q9 direction order is the paper's (Sec. 2.1): e_0 = (0,0), (1,0), (0,1), (-1,0),
 *    (0,-1), (1,1), (-1,1), (-1,-1), (1,-1).
 */
#ifndef MLBM_H
#define MLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLBM_OK 0
#define MLBM_EINVAL (-1)    /* bad argument, size or state                         */
#define MLBM_ENOMEM (-2)    /* host or device allocation failed                    */
#define MLBM_ECUDA (-3)     /* CUDA runtime error or no usable device              */
#define MLBM_ESINGULAR (-4) /* a collocation matrix was singular / failed checks   */
#define MLBM_ETIMEOUT (-5)  /* a bounded wait ran out                              */

#define MLBM_GEOM_PERIODIC 0 /* periodic box [0,lx) x [0,ly), minimum-image distances */
#define MLBM_GEOM_ANNULUS 1  /* ring r_in <= |x| <= r_out centred at the origin         */

#define MLBM_STENCIL_OWN 0     /* one stencil per node for all directions (default)        */
#define MLBM_STENCIL_NEAREST 1 /* stencil of the node nearest to each departure point      */

#define MLBM_F32 32 /* FP32 deviation storage, FP32 arithmetic */
#define MLBM_F64 64 /* FP64 populations, FP64 arithmetic       */

/* mlbm_build_weights flags */
#define MLBM_KEEP_W32 1 /* keep FP32 shape vectors on the device (needed by MLBM_F32 steps) */
#define MLBM_KEEP_W64 2 /* keep FP64 shape vectors on the device (needed by MLBM_F64 steps) */

typedef struct mlbm_cloud mlbm_cloud;
typedef struct mlbm_weights mlbm_weights;

/* One independent simulation ("segment") of a cloud.  Several segments batch independent
 * runs of uneven size, stencil and degree into the same launches. */
typedef struct {
    int geometry;        /* MLBM_GEOM_PERIODIC or MLBM_GEOM_ANNULUS                          */
    double lx, ly;       /* periodic box edge lengths (physical units)                       */
    double r_in, r_out;  /* annulus wall radii (physical units)                              */
    int k;               /* stencil size N_L, centre included (Sec. 2.2)                     */
    int degree;          /* total degree d of the polynomial augmentation (eq. poly_sets)    */
    double dx_ml;        /* streaming distance dx_ml (Sec. 2.3), physical units; in lattice
                            units it is 1, so c_k = e_k and the departure point of population
                            k at node i is x_i - e_k dx_ml                                     */
    int stencil_mode;    /* MLBM_STENCIL_OWN: population k of node i is interpolated in node
                            i's own stencil, shared by all directions; MLBM_STENCIL_NEAREST:
                            in the stencil of the Eulerian node nearest to its departure point
                            (Sec. 2.3 and the appendix algorithm), which lets dx_ml exceed the
                            node spacing                                                       */
} mlbm_segment_desc;

/* Per-segment step parameters, lattice units. */
typedef struct {
    double tau;  /* BGK relaxation time (eq. LBM_collision), > 0.5                          */
    double g;    /* body-force magnitude (Sec. 3 forcing term omega_k e_k.g / c_s^2); the
                    direction is azimuthal (-sin phi, cos phi) on an annulus and +x in a
                    periodic box; 0 disables the force                                        */
    double rho0; /* reference density of the FP32 deviation storage                          */
} mlbm_params;

/* Message describing the last failure on the calling thread ("" if none). */
const char *mlbm_last_error(void);

/* Library ABI version (increments when entry points are added or changed). */
int mlbm_abi_version(void);

/* ---------------------------------------------------------------------------------------
 * mlbm_build_cloud -- stencil build, host side (Sec. 2.2, Sec. 3 periodic stencil search,
 * Sec. 3 annulus wall bounce-back; set-up loop of the appendix algorithm).
 *
 *   xy           host, [2][n] float64: x coordinates then y coordinates, original order.
 *   n            total node count over all segments (>= 1).
 *   segs         host, nseg descriptors.
 *   seg_offsets  host, nseg + 1 int64: segment s owns original nodes
 *                [seg_offsets[s], seg_offsets[s+1]); seg_offsets[0] = 0, seg_offsets[nseg] = n.
 *   nseg         >= 1.
 *   out          receives a library-owned cloud (free with mlbm_cloud_free).
 *
 * Per segment: Morton reorder; N_L nearest neighbours of every node by (squared distance,
 * original index) ascending, the node itself first, minimum-image distances in a periodic
 * box; the bounce-back mask (bit k set when the departure point of population k leaves the
 * annulus, relative tolerance 1e-12 on r^2); the force direction; the transposed stencil
 * used by the adjoint.  Errors: MLBM_EINVAL (k > segment size, k < number of monomials,
 * bad geometry or offsets, N_L * N >= 2^31), MLBM_ENOMEM.
 * ------------------------------------------------------------------------------------- */
int mlbm_build_cloud(const double *xy, int64_t n, const mlbm_segment_desc *segs,
                     const int64_t *seg_offsets, int nseg, mlbm_cloud **out);
void mlbm_cloud_free(mlbm_cloud *cloud);

/* ---------------------------------------------------------------------------------------
 * mlbm_build_cloud_device -- the same stencil build on the GPU (Sec. 2.2 stencils, Sec. 2.3
 * departure nodes, Sec. 3 periodic search and bounce-back): Morton codes and a stable radix
 * sort, a bucket grid and one thread per N_L-nearest-neighbour query, departure nodes, masks,
 * force directions and the transposed stencil, all in kernels.
 *
 *   xy, n, segs, seg_offsets, nseg, out   as mlbm_build_cloud (xy is a host pointer).
 *   stream   CUDA stream for the build; the call synchronises it before returning.
 *
 * The result is identical, array for array and bit for bit, to mlbm_build_cloud on the same
 * arguments: every distance that decides a rank is rounded as the host build rounds it.
 * Device memory: about 8 (N_L + 10) bytes per node, freed before returning.
 * Errors: as mlbm_build_cloud, plus MLBM_ECUDA (no device, launch failure) and MLBM_ENOMEM
 * (device allocation).
 * ------------------------------------------------------------------------------------- */
int mlbm_build_cloud_device(const double *xy, int64_t n, const mlbm_segment_desc *segs,
                            const int64_t *seg_offsets, int nseg, void *stream, mlbm_cloud **out);


/* Total node count N of a cloud (-1 if cloud is NULL). */
int64_t mlbm_cloud_size(const mlbm_cloud *cloud);

/* perm (host, n int64): perm[p] = original index of the node at stored position p. */
int mlbm_cloud_perm(const mlbm_cloud *cloud, int64_t *perm);

/* Stencil of segment seg in original numbering relative to the segment start:
 * idx (host, [N_L][n_seg] int32), idx[j * n_seg + i] = member j of node i's stencil,
 * i in original segment order. */
int mlbm_cloud_stencil(const mlbm_cloud *cloud, int seg, int32_t *idx);

/* Departure nodes of segment seg: near (host, [8][n_seg] int32), near[(k-1) * n_seg + i] =
 * the node (original numbering relative to the segment start) whose stencil interpolates
 * population k of node i, i in original segment order: the node nearest to x_i - e_k dx_ml by
 * (squared distance, original index) in MLBM_STENCIL_NEAREST mode, i itself in
 * MLBM_STENCIL_OWN mode. */
int mlbm_cloud_departure_nodes(const mlbm_cloud *cloud, int seg, int32_t *near);

/* Bounce-back mask of all nodes in original order: mask (host, n uint16), bit k (1..8)
 * set when population k of the node is an unknown wall population. */
int mlbm_cloud_bounce_mask(const mlbm_cloud *cloud, uint16_t *mask);

/* ---------------------------------------------------------------------------------------
 * mlbm_build_weights -- RBF-FD shape vectors on the GPU, FP64 (Sec. 2.2 eq. shape_vector,
 * Sec. 2.3 basis r^3 + P_d, LU with partial pivoting; set-up loop of the appendix
 * algorithm).
 *
 * For every node the collocation matrix Phi_L = [[R, P], [P^T, 0]] of its own stencil is
 * assembled in coordinates centred on the node and divided by the stencil radius,
 * factorised once by LU with partial pivoting, and solved for the eight right-hand sides
 * phi_L(x_i - e_k dx_ml), k = 1..8 (the rest population needs no interpolation: its
 * departure point is the node itself).  The first N_L solution entries are the shape
 * vector.  One batched kernel solves all systems of all segments (uneven sizes allowed).
 *
 *   cloud    a cloud from mlbm_build_cloud (not modified; may be freed afterwards).
 *   flags    MLBM_KEEP_W32 and/or MLBM_KEEP_W64 (0 means both).
 *   stream   CUDA stream; the call synchronises it before returning.
 *   out      receives the library-owned device weights object (free with
 *            mlbm_weights_free).  It holds the stencil, shape vectors, masks, force
 *            directions, the transposed stencil and the cached CUDA graphs.
 *   n_bad    host, optional: number of systems that were singular (|pivot| <= 1e-14 max|Phi|)
 *            or failed the polynomial-reproduction check (max error > 1e-8).
 * Errors: MLBM_ESINGULAR if n_bad > 0 (the object is still returned, bad shape vectors are
 * zero), MLBM_ECUDA, MLBM_ENOMEM, MLBM_EINVAL.
 * ------------------------------------------------------------------------------------- */
int mlbm_build_weights(const mlbm_cloud *cloud, int flags, void *stream, mlbm_weights **out,
                       int64_t *n_bad);
void mlbm_weights_free(mlbm_weights *w);

/* Number of segments and total nodes of a weights object. */
int mlbm_weights_info(const mlbm_weights *w, int64_t *n_nodes, int *nseg);

/* Copy the FP64 shape vectors of segment seg to the host: W (host, [8][N_L][n_seg]
 * float64), W[((k-1) * N_L + j) * n_seg + i] for direction k = 1..8, stencil member j as
 * in mlbm_cloud_stencil, node i in original segment order.  Needs MLBM_KEEP_W64. */
int mlbm_weights_download(const mlbm_weights *w, int seg, double *W);

/* Copy the FP32 shape vectors the FP32 step uses to the host: W (host, float32, the layout of
 * mlbm_weights_download).  Entries j >= 1 are the FP64 values rounded one by one so that the
 * reproduction of the monomials of degree 1..min(d, 6) about the stencil centre (Sec. 2.2,
 * the P^T block of eq. rbf_interp_set_augmented) holds as closely as FP32 allows, each within
 * 2^-12 max|w| of its FP64 value; entry 0 (the centre, which the FP32 difference form does not
 * read) is the FP64 value rounded to nearest.  Needs MLBM_KEEP_W32. */
int mlbm_weights_download_f32(const mlbm_weights *w, int seg, float *W);

/* Replace the shape vectors of segment seg with caller-supplied FP64 values (same layout as
 * mlbm_weights_download); the FP64 copy and the FP32 copy rounded from it are overwritten.  idx
 * (host, [N_L][n_seg] int32, layout of mlbm_cloud_stencil) must equal the library's own
 * stencil, else MLBM_EINVAL and nothing changes.  Synchronous; the adjoint's coefficients,
 * if built, are discarded (after a device synchronisation) and rebuilt from the new shape
 * vectors on the next mlbm_adjoint_step. */
int mlbm_weights_upload(mlbm_weights *w, int seg, const double *W, const int32_t *idx);

/* ---------------------------------------------------------------------------------------
 * mlbm_init -- initial state (Sec. 3 initial condition; set-up loop of the appendix
 * algorithm): f_k = f^eq_k(rho, u) (eq. feq), stored as its post-collision value, which for
 * an equilibrium is f^eq_k plus the forcing term omega_k e_k.g / c_s^2.
 *
 *   params   host, nseg parameter sets.
 *   dtype    MLBM_F32 or MLBM_F64.
 *   rho, ux, uy  device, n float64 each, ORIGINAL order.
 *   f_out    device, [9][N] of dtype, stored order.
 * ------------------------------------------------------------------------------------- */
int mlbm_init(const mlbm_weights *w, const mlbm_params *params, int dtype, const double *rho,
              const double *ux, const double *uy, void *f_out, void *stream);

/* ---------------------------------------------------------------------------------------
 * mlbm_step -- one time step of all segments in one fused launch (appendix algorithm
 * COLLIDE/STREAM reordered as a pull; Sec. 2.3 semi-Lagrangian streaming; Sec. 3 wall
 * bounce-back and forcing):
 *   1. fhat_k(i) = sum_j W_k[j](i) f^post_k(s_j(i)), k = 1..8; fhat_0(i) = f^post_0(i);
 *   2. fhat_k(i) = fhat_k'(i) (streamed values) where bit k of the bounce-back mask is set;
 *   3. rho, u of fhat (eq. macro_var); f^post = fhat - (fhat - f^eq)/tau + omega_k e_k.g/c_s^2.
 *
 *   params   host, nseg parameter sets (tau > 0.5 required).
 *   dtype    MLBM_F32 (needs MLBM_KEEP_W32 weights) or MLBM_F64 (needs MLBM_KEEP_W64).
 *   f_in     device, [9][N] dtype, stored order: post-collision state of level n.
 *   f_out    device, [9][N] dtype: post-collision state of level n+1.  Must not alias f_in.
 *   moments  device, optional (NULL = skip): [3][N] of dtype, stored order, receives
 *            rho, u_x, u_y of fhat (the macroscopic fields of level n+1).
 * ------------------------------------------------------------------------------------- */
int mlbm_step(const mlbm_weights *w, const mlbm_params *params, int dtype, const void *f_in,
              void *f_out, void *moments, void *stream);

/* nsteps steps ping-ponging between two state buffers: step 1 reads f_a and writes f_b,
 * step 2 reads f_b and writes f_a, ...  The result is in f_a when nsteps is even, else in
 * f_b.  The step sequence is captured once into a CUDA graph (cached in the weights object
 * per buffers, dtype and parameters) and replayed.  Calls on one weights object must not
 * run concurrently from several host threads. */
int mlbm_run(mlbm_weights *w, const mlbm_params *params, int dtype, void *f_a, void *f_b,
             int64_t nsteps, void *stream);

/* Each segment run for its own number of steps in one call (the batched convergence sweep,
 * whose runs end at different times, e.g. the paper's end time of each resolution, Sec. 3).
 *   seg_steps  host, nseg int64 >= 0: steps of each segment.
 * The call makes S = max(seg_steps) steps ping-ponging between f_a and f_b as mlbm_run does,
 * each step over the tiles of the segments not yet done (in CUDA graphs per run of steps with
 * the same active segments), and then copies the final state of every segment whose count
 * has the other parity than S into the result buffer: the result (every segment after its
 * own number of steps) is in f_a when S is even, else in f_b.  Finished segments are not
 * touched otherwise, so each segment's result equals a run of that segment alone.  The other
 * buffer holds scratch.  Calls on one weights object must not run concurrently.
 * Errors: MLBM_EINVAL (NULL, f_a == f_b, negative count), MLBM_ENOMEM, MLBM_ECUDA. */
int mlbm_run_until(mlbm_weights *w, const mlbm_params *params, int dtype, void *f_a, void *f_b,
                   const int64_t *seg_steps, void *stream);

/* ---------------------------------------------------------------------------------------
 * mlbm_step_host -- one time step (as mlbm_step) for each of nbatch independent states held
 * in HOST memory, end to end: state b is copied to the device, stepped, and its new
 * post-collision state copied back.  Two device buffers per direction and one copy stream per
 * direction let the copy in of state b + 1 and the copy out of state b - 1 run while state b
 * steps, so the call is bound by the slower of the host link and the step.
 *
 *   w, params, dtype   as mlbm_step.
 *   nbatch   number of states (>= 1).
 *   f_in     host, nbatch pointers, each to a [9][N] state of dtype in stored order.
 *   f_out    host, nbatch pointers receiving the stepped states; f_out[b] may equal f_in[b]
 *            but must not overlap f_in[c] for c != b.  Inputs may repeat; outputs that
 *            overlap each other end up holding the later state.
 *   stream   CUDA stream the steps run on (the copies start after work already queued on it);
 *            every copy and step has finished when the call returns.
 * Page-locked host memory (cudaHostAlloc, cudaHostRegister) lets the copies run
 * asynchronously; pageable memory gives the same results with serialised copies.  Device
 * memory: four state buffers kept in the weights object for later calls.
 * Errors: MLBM_EINVAL, MLBM_ENOMEM, MLBM_ECUDA.
 * ------------------------------------------------------------------------------------- */
int mlbm_step_host(mlbm_weights *w, const mlbm_params *params, int dtype, int64_t nbatch,
                   const void *const *f_in, void *const *f_out, void *stream);

/* ---------------------------------------------------------------------------------------
 * mlbm_sc_step -- one time step of the Shan-Chen single-component multiphase model on the
 * meshless cloud (the extension the paper's discussion names: the particle interactions sit
 * in the local collision; the model is Shan & Chen 1993, the paper gives no formulas):
 *   1. streaming as mlbm_step: fhat_k(i) = sum_j W_k[j](i) f^post_k(s_j(i));
 *   2. psi_i = rho_psi (1 - exp(-rho_i / rho_psi)) of the density of fhat;
 *   3. F_i = -G psi_i sum_k omega_k psi(x_i + e_k dx_ml) e_k, psi at x_i + e_k dx_ml (the
 *      departure point of the opposite direction) interpolated with the streaming's own
 *      shape vectors, in the stencil that interpolates that departure point (the node's own,
 *      or under MLBM_STENCIL_NEAREST that of the point's nearest node);
 *   4. BGK collision of fhat towards f^eq(rho, u + tau F / rho), plus the body force term of
 *      mlbm_step.
 *
 *   w          weights of periodic segments (no walls: MLBM_EINVAL otherwise; a wall would
 *              need a value of psi beyond it, a wetting choice), either stencil rule.
 *   params     host, nseg parameter sets as mlbm_step (tau, body force g, rho0).
 *   sc         host, nseg pairs {G, rho_psi}: coupling (with rho_psi = 1, G < -4 separates
 *              phases) and the density scale of psi (> 0).
 *   dtype, f_in, f_out, moments, stream   as mlbm_step; moments are those of fhat (before
 *              the velocity shift).
 * Two launches per step (stream + psi, then force + collision); a psi scratch of N doubles is
 * kept in the weights object.  Errors: MLBM_EINVAL, MLBM_ENOMEM, MLBM_ECUDA.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    double G;       /* interaction strength */
    double rho_psi; /* density scale of the pseudopotential */
} mlbm_sc_params;

int mlbm_sc_step(mlbm_weights *w, const mlbm_params *params, const mlbm_sc_params *sc, int dtype,
                 const void *f_in, void *f_out, void *moments, void *stream);

/* ---------------------------------------------------------------------------------------
 * mlbm_moments -- macroscopic fields (eq. macro_var) of the time level whose post-collision
 * state is f: rho = sum f, rho u = sum f e - g (collision conserves rho and adds exactly the
 * body force g to rho u, so these are the post-streaming moments the paper reports).
 *
 *   f             device, [9][N] dtype, stored order.
 *   rho, ux, uy   device, n float64 each, ORIGINAL order.
 * ------------------------------------------------------------------------------------- */
int mlbm_moments(const mlbm_weights *w, const mlbm_params *params, int dtype, const void *f,
                 double *rho, double *ux, double *uy, void *stream);

/* ---------------------------------------------------------------------------------------
 * mlbm_norms -- the sums behind the normalised L2 error of eq. (L2norm) and the relative
 * velocity residual of the Sec. 3 stopping rule, reduced deterministically (fixed order,
 * two passes) on the device:
 *   out[0] = sum_i (a_i - b_i)^2 + (c_i - d_i)^2,  out[1] = sum_i b_i^2 + d_i^2,
 *   out[2] = sum_i a_i^2 + c_i^2.
 *   a, b, c, d   device, n float64 each (c and d may both be NULL: single component).
 *   out          host, 3 float64.  The call synchronises the stream.
 * ------------------------------------------------------------------------------------- */
int mlbm_norms(const mlbm_weights *w, const double *a, const double *b, const double *c,
               const double *d, int64_t n, double *out, void *stream);

/* ---------------------------------------------------------------------------------------
 * Standard lattice LBM (Sec. 2.1, eq. LBM_streaming): nodes on a periodic nx x ny lattice with
 * spacing dx_ml, streaming as the index shift f_k(x) <- f^post_k(x - e_k), the same BGK
 * collision, forcing (direction +x) and state conventions as the meshless step.  The paper
 * compares the meshless method with it; it is also the limit the meshless step reduces to
 * when the nodes form that lattice.  Node index iy * nx + ix; no weights object is needed.
 *
 * mlbm_lattice_init: f_out (device, [9][nx*ny] dtype) = equilibrium at rho, ux, uy (device,
 *   nx*ny float64 each) plus the forcing term, as mlbm_init.
 * mlbm_lattice_step: one step f_in -> f_out (must not alias); moments (device, optional,
 *   [3][nx*ny] dtype) receives rho, u_x, u_y of the streamed populations.
 * params points to ONE parameter set.  Errors: MLBM_EINVAL (sizes, tau <= 1/2, dtype), MLBM_ECUDA.
 * ------------------------------------------------------------------------------------- */
int mlbm_lattice_init(int64_t nx, int64_t ny, const mlbm_params *params, int dtype,
                      const double *rho, const double *ux, const double *uy, void *f_out,
                      void *stream);
int mlbm_lattice_step(int64_t nx, int64_t ny, const mlbm_params *params, int dtype,
                      const void *f_in, void *f_out, void *moments, void *stream);

/* ---------------------------------------------------------------------------------------
 * mlbm_norms_noalloc -- the sums of mlbm_norms computed without allocating any memory.  The
 * paper has no counterpart; this is a library facility.
 *
 * Some callers cannot call cudaMalloc: code that runs while a memory pool owns the device
 * (a framework's caching allocator that has reserved the free memory, where an extra
 * cudaMalloc fails or fragments the pool), latency-critical loops that cannot afford the
 * implicit device synchronisation of cudaMalloc / cudaFree, and monitoring code that must not
 * change the process's memory footprint.  mlbm_norms needs a weights object whose scratch it
 * allocates on first use; this variant needs no weights object and calls no allocating
 * routine (no cudaMalloc, cudaFree or library allocator).  Its scratch is a fixed array of
 * 4096 x 3 doubles (96 KiB) in the library's own device memory, which every GPU that loads the
 * library holds until the process exits.
 *
 *   a, b, c, d  device, n float64 each (c and d may both be NULL: single component)
 *   n           0 <= n <= 16,777,216 (4096 blocks of 4096 elements); larger n returns
 *               MLBM_EINVAL with a message naming the limit, and nothing is launched
 *   out         device, 3 float64: the same three sums as mlbm_norms (summed in a different
 *               block order, so equal to rounding, not bitwise)
 * The call is stream-ordered and asynchronous (it does not synchronise).  The first call on
 * each device looks up the scratch array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture on the device.  The
 * address is kept for the life of the process: after a cudaDeviceReset (which recreates the
 * device's context and reloads the library's device code) it is stale, so do not use this
 * entry point across a device reset.  All calls share the one array and it keeps the last
 * call's partial sums: calls that overlap on the GPU (different streams or host threads
 * without ordering) race and give wrong results.
 * Errors: MLBM_EINVAL, MLBM_ECUDA.
 * ------------------------------------------------------------------------------------- */
int mlbm_norms_noalloc(const double *a, const double *b, const double *c, const double *d,
                       int64_t n, double *out, void *stream);

/* ---------------------------------------------------------------------------------------
 * Adjoint (discrete reverse mode of the step above).  With s^{n+1} = Step(s^n; tau, g):
 *
 * mlbm_adjoint_step: given lam_next = dL/ds^{n+1}, writes lam_prev = dL/ds^n (the transpose
 * of the linearised step: collision Jacobian including d f^eq / d(rho, u), bounce-back
 * transpose, then the transpose of the interpolation done as a deterministic pull over the
 * transposed stencil) and adds dL/dtau and dL/dg of this step to grad (device, 2 * nseg
 * float64, [seg][tau, g]).  s_prev is the forward state s^n (device, [9][N] dtype).
 * s_next is optional (NULL allowed): the forward's output s^{n+1} = Step(s^n) with the same
 * weights and params.  The Jacobian and dL/dtau need the moments and the non-equilibrium part
 * of the interpolated populations fhat; with s_next they are taken from it (the collision
 * keeps rho, adds g to rho u and scales fhat - f^eq by 1 - 1/tau), which skips re-reading the
 * shape vectors; without it, or when |1 - 1/tau| < 1/16 in any segment (fhat is not
 * recoverable near tau = 1), fhat is recomputed from s_prev.  Both routes agree to rounding.
 * lam_next and lam_prev: device [9][N] dtype; lam_prev must alias neither lam_next nor s_next.
 * Both stencil rules: under MLBM_STENCIL_NEAREST the transposed interpolation runs over the
 * nodes whose departure-node stencils hold each node.  A weights object with any
 * MLBM_STENCIL_NEAREST segment needs s_next and |1 - 1/tau| >= 1/16 in every segment (else
 * MLBM_EINVAL, nothing launched).  The first call builds the transposed tables (host work and
 * a device copy of the departure nodes, then kept with the weights).
 * ------------------------------------------------------------------------------------- */
int mlbm_adjoint_step(const mlbm_weights *w, const mlbm_params *params, int dtype,
                      const void *s_prev, const void *s_next, const void *lam_next,
                      void *lam_prev, double *grad, void *stream);

/* Seed of the reverse sweep for a loss on the macroscopic fields of the level whose
 * post-collision state is f (the outputs of mlbm_moments): given drho, dux, duy (device,
 * n float64, ORIGINAL order) = dL/d(rho, u_x, u_y), writes lam = dL/df (device, [9][N]
 * dtype) and adds the explicit dependence on g to grad. */
int mlbm_moments_adjoint(const mlbm_weights *w, const mlbm_params *params, int dtype,
                         const void *f, const double *drho, const double *dux,
                         const double *duy, void *lam, double *grad, void *stream);

/* End of the reverse sweep through mlbm_init: given lam0 = dL/ds^0 (device [9][N] dtype),
 * writes drho, dux, duy = dL/d(rho, u_x, u_y) of the initial fields (device, n float64,
 * ORIGINAL order; rho, ux, uy are the initial fields) and adds the forcing term's
 * dependence on g to grad. */
int mlbm_init_adjoint(const mlbm_weights *w, const mlbm_params *params, int dtype,
                      const double *rho, const double *ux, const double *uy, const void *lam0,
                      double *drho, double *dux, double *duy, double *grad, void *stream);

/* ---------------------------------------------------------------------------------------
 * mlbm_fp64_fma_rate -- a measurement facility with no counterpart in the paper: enqueues a
 * kernel of independent FP64 fused multiply-add chains (16 per thread, 256 threads per CTA,
 * blocks_per_sm CTAs on every SM, iters FMAs per chain) on `stream` and returns through
 * *flops (host) the floating-point operations it performs (2 per FMA).  Timed by the caller
 * (CUDA events on the same stream), flops / time is the device's sustained FP64 rate, the
 * denominator for kernels bound by FP64 arithmetic.
 *   sink      device, at least blocks_per_sm * (number of SMs) float64 (one sum per CTA,
 *             written so that the work is not optimised away; caller-owned)
 *   sink_len  its length; too short returns MLBM_EINVAL with nothing launched
 * Asynchronous.  Errors: MLBM_EINVAL, MLBM_ECUDA.
 * ------------------------------------------------------------------------------------- */
int mlbm_fp64_fma_rate(int64_t iters, int blocks_per_sm, double *sink, int64_t sink_len,
                       void *stream, double *flops);

#ifdef __cplusplus
}
#endif

#endif /* MLBM_H */

/*
 * mlpg.h - C ABI of the GB300 (sm_103a) library for the time-dependent
 * discrete-ordinates transport solve on a meshless MLPG discretisation with
 * reproducing-kernel (RK) functions integrated over Voronoi-like cells
 * (Bassett & Owen, arXiv 2008.02205).
 *
 * Call order: mlpg_create -> mlpg_integrate -> mlpg_assemble -> mlpg_step* ->
 * mlpg_scalar_flux; mlpg_destroy at any time.  A call out of order returns
 * MLPG_ERR_STATE.  No call aborts or throws: each returns a status and, on
 * failure, mlpg_last_error() describes it.  Inputs are copied at create; the
 * caller keeps ownership of every pointer it passes.  Host-pointer variants
 * copy directly from or to the caller's (pageable or pinned) memory on the
 * library stream and return once the copy is complete; `_dev` variants take
 * device pointers valid on the device that was current at create.
 *
 * All arrays are row-major.  Angular fluxes use the layout psi[i][m] (point i,
 * direction m; the direction index varies fastest).
 */
#ifndef MLPG_H
#define MLPG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlpg_ctx mlpg_ctx; /* opaque, owned by the library */

typedef enum {
    MLPG_OK = 0,
    MLPG_ERR_ARG = -1,           /* invalid argument (null pointer, bad size, bad enum) */
    MLPG_ERR_STATE = -2,         /* call out of order */
    MLPG_ERR_OOM = -3,           /* device or host allocation failed */
    MLPG_ERR_CUDA = -4,          /* CUDA runtime error (message in mlpg_last_error) */
    MLPG_ERR_GEOMETRY = -5,      /* a cell could not be built (point outside the box, ...) */
    MLPG_ERR_RK_SINGULAR = -6,   /* an RK moment matrix is singular: too few neighbours */
    MLPG_ERR_NOT_CONVERGED = -7  /* a Krylov solve hit its iteration cap */
} mlpg_status;

typedef enum {
    MLPG_FP64 = 0,  /* every step in FP64 */
    MLPG_MIXED = 1  /* FP32 operator streams and Krylov vectors; FP64 RK inversion,
                       Arnoldi scalars, Hessenberg least squares and step residuals
                       (iterative refinement of each backward-Euler step) */
} mlpg_precision;

typedef struct {
    int dim;               /* spatial dimension: 2 (polygonal cells) or 3 (polyhedral cells); default 2 */
    double lo[3], hi[3];   /* axis-aligned box domain */
    double tau_factor;     /* SUPG tau_i = tau_factor * h_i, h_i = R_i / 2 (Sec. 4.1); default 1 */
    double c;              /* speed of light in 1/(c dt) (Sec. 4.1); default 1 */
    int precision;         /* mlpg_precision; default MLPG_FP64 */
    double inner_tol;      /* per-direction transport GMRES: ||r|| <= tol ||b||; default 1e-12 */
    double outer_tol;      /* scattering GMRES on Phi (Eq. krylov-operator); default 1e-12 */
    int inner_restart;     /* inner GMRES restart length (<= 32); default 20 (FP64), mixed_restart in MLPG_MIXED */
    int outer_restart;     /* outer GMRES restart length (<= 32); default 30 */
    int max_inner;         /* inner iteration cap per solve; default 2000 */
    int max_outer;         /* outer iteration cap per solve; default 500 */
    double refine_tol;     /* MLPG_MIXED: FP64 step residual ||R|| <= tol ||f||; default 1e-11 */
    int max_refine;        /* MLPG_MIXED: refinement sweeps per step; default 12 */
    double mixed_inner_tol;/* MLPG_MIXED: tolerance of the FP32 correction solves; default 1e-2 */
    int check_every;       /* inner GMRES: host convergence check interval (steps); default 3 */
    int mixed_restart;     /* MLPG_MIXED: restart length of the FP32 inner GMRES (<= 32); default 20.
                              The FP32 correction solves keep the iterate reached at their iteration
                              caps (max_inner; one outer restart cycle): the FP64 step residual alone
                              decides convergence (MLPG_ERR_NOT_CONVERGED after max_refine sweeps) */
    int mixed_reorth;      /* MLPG_MIXED: Gram-Schmidt passes in the FP32 inner GMRES: 1 = classical
                              Gram-Schmidt with one re-orthogonalisation (CGS2), 0 = a single
                              classical pass; the FP64 solves always use CGS2; default 0 */
    int mixed_half_prec;   /* MLPG_MIXED: 1 = the FP32 correction solves use the block-Jacobi
                              inverses stored in FP16 (scaled by a power of two per block and
                              direction), 0 = FP32 inverses; default 1 */
    int outer_method;      /* scattering solve: 0 = GMRES on Phi (Eq. krylov-operator), 1 = source
                              iteration Phi <- b_phi + D L^-1 MS Phi, stopped when the update is
                              below outer_tol of Phi (max_outer iterations); default 0 */
    int rk_order;          /* order of the RK correction (Sec. 2.2): 0 (constants reproduced),
                              1 (linear) or 2 (quadratic; needs kernels spanning at least five
                              neighbours, e.g. extent 2.5-3 point spacings); 3D: 0 or 1;
                              default 1 */
    void *stream;          /* cudaStream_t to run on; NULL = a stream owned by the library */
    int apply_kernel;      /* MLPG_MIXED batched L-apply: 0 = automatic (m % 4 == 0: row tiles with a
                              staged halo when that takes at most two direction chunks, else row
                              tiles in gather mode; otherwise row teams), 1 = one team of
                              direction lanes per row gathering X through L1, 2 = row tiles with the
                              tile's neighbour rows staged in shared memory (m % 4 == 0), 3 = the
                              same tiles with the combination of the base arrays on tensor cores
                              (TF32 split in high and low parts: FP32 accuracy; m % 8 == 0),
                              4 = row tiles with only the operator records staged and X read
                              from global memory (L2) per entry: no halo in shared memory, so a
                              chunk holds all directions (m % 4 == 0; for large direction sets,
                              e.g. 3D, whose halos leave room for few directions per chunk);
                              default 0 */
    int tile_rows;         /* row tiles: rows per tile, 32 or 64 (apply_kernel 2, 3), 4, 8, 16 or
                              32 (apply_kernel 4); 0 = 64, or in gather mode the most rows that
                              keep a CTA at or below 320 threads */
    int tile_dpt;          /* row tiles: directions per thread, 4 or 8 (must divide m); 0 = 8 when
                              m % 8 == 0 with a staged halo, else 4 */
    int outer_precond;     /* outer GMRES on Phi: 0 = none (the paper's), 1 = DSA-like diffusion
                              correction, right preconditioner I + C^-1 Ms with the P1-diffusion
                              operator C = diag(1/(3 sigma_t,i)) sum_a K_aa + kappa M0 + Mt - Ms
                              + 1/2 sum_f S_f built from the integrated forms (Sec. 5.3 and Sec. 6
                              name diffusion acceleration without deriving one); the outer GMRES is
                              then flexible; needs outer_method 0; default 0 */
    double dsa_tol;        /* outer_precond 1: tolerance of the FP64 diffusion solves; default 1e-10 */
    int dsa_max;           /* outer_precond 1: iteration cap of a diffusion solve (its iterate is
                              kept at the cap); default 500 */
    int cells_3d;          /* 3D cells (Sec. 3.1) built 0 = on the device (one thread per cell),
                              1 = on the host cores; both give the same cells; default 0 */
} mlpg_options;

typedef struct {
    int64_t n, nnz;              /* points, overlap-pattern entries */
    int32_t m;                   /* directions */
    int64_t n_volume_qp;         /* volume quadrature points (Sec. 3.2) */
    int64_t n_boundary_qp;       /* boundary quadrature points */
    int32_t steps;               /* backward-Euler steps taken */
    int32_t last_outer_iters;    /* scattering GMRES iterations, last step (summed over refinements) */
    int64_t last_inner_iters;    /* inner GMRES iterations summed over directions and solves, last step */
    int32_t last_inner_solves;   /* batched L^{-1} applications in the last step */
    int32_t last_refinements;    /* MLPG_MIXED: refinement sweeps in the last step */
    double last_residual;        /* final relative step residual (FP64) of the last step */
    int64_t total_outer_iters, total_inner_iters;
    int64_t spmm_launches;       /* batched L-apply launches since create */
    double spmm_ms;              /* their device time (when timing is enabled), ms */
    int64_t spmm_bytes;          /* algorithmic bytes of one batched L-apply (active precision) */
    int64_t kernel_launches;     /* kernels this context launched since create */
    int64_t device_bytes;        /* device memory this context holds (its own allocations) */
    int32_t apply_kernel;        /* FP32 batched L-apply in use once operators exist: 1 row teams,
                                    2 row tiles, 3 row tiles on tensor cores, 4 row tiles gathering
                                    X from global memory (see
                                    mlpg_options.apply_kernel); 0 before */
    int32_t tile_chunk;          /* row tiles: directions per CTA (the chunk), 0 otherwise */
    int64_t tile_max_halo;       /* row tiles: largest halo (staged neighbour rows) of a tile */
    int64_t last_dsa_iters;      /* outer_precond 1: diffusion-solve iterations, last step */
    int64_t total_dsa_iters;
} mlpg_stats;

/* Default options (values listed in mlpg_options); a NULL opt is ignored.  A
 * library service with no paper counterpart. */
void mlpg_default_options(mlpg_options *opt);

/* Create a problem (Sec. 4.1, Eq. transport-equation with the discrete
 * ordinates of Sec. 4.1):
 *   points[n*dim]        point positions x_i (inside the box)
 *   kernel_extent[n]     kernel support radius R_i (cubic spline, h_i = R_i/2)
 *   omega[m*3], w[m]     ordinates Omega_m (unit vectors) and weights, sum w = 4 pi
 *   sigma_t[n], sigma_s[n], q[n]
 *                        total / scattering cross sections and isotropic source
 *                        per steradian, constant over each point's cell
 * Host pointers.  Fails with MLPG_ERR_ARG on bad sizes, non-finite values,
 * non-positive extents or non-unit ordinates, MLPG_ERR_GEOMETRY for a point
 * outside the box.  *out is NULL when the options or sizes are rejected; a
 * failure after that (a bad value, a CUDA or allocation error) leaves in *out
 * a context that holds the message for mlpg_last_error() and must be passed
 * to mlpg_destroy.  */
mlpg_status mlpg_create(const mlpg_options *opt, int64_t n, const double *points,
                        const double *kernel_extent, int32_t m, const double *omega,
                        const double *w, const double *sigma_t, const double *sigma_s,
                        const double *q, mlpg_ctx **out);

/* Same as mlpg_create with every array a device pointer (readable from the
 * device current at this call); the same checks, errors and *out contract. */
mlpg_status mlpg_create_dev(const mlpg_options *opt, int64_t n, const double *points,
                            const double *kernel_extent, int32_t m, const double *omega,
                            const double *w, const double *sigma_t, const double *sigma_s,
                            const double *q, mlpg_ctx **out);

/* Incoming isotropic angular flux psi_b on box face `face` (0:-x 1:+x 2:-y
 * 3:+y, in 3D also 4:-z 5:+z), Eq. rad-boundary.  Default 0 (vacuum).  Any
 * state after create; takes effect at the next step.  MLPG_ERR_ARG for a face
 * outside [0, 2 dim) or a non-finite psi_b. */
mlpg_status mlpg_set_inflow(mlpg_ctx *ctx, int face, double psi_b);

/* Initial angular flux coefficients Psi_i(0) = psi_init(x_i) (Sec. 4.1), host
 * psi0[n*m] in [i][m] layout (the caller guarantees n*m values); NULL = 0.
 * Any state after create.  Also clears the step history the mixed-precision
 * predictor extrapolates from. */
mlpg_status mlpg_set_initial(mlpg_ctx *ctx, const double *psi0);

/* Neighbour search (Sec. 3.4, overlap connectivity), Voronoi-like cells and
 * their quadrature points (Sec. 3.1-3.2, App. A; 2D cells clipped on the
 * device, 3D cells on the host cores), RK point interpolation at the centres
 * (Eq. flux-expansion).  MLPG_ERR_RK_SINGULAR if an RK moment matrix is
 * singular, MLPG_ERR_GEOMETRY if a cell is empty, MLPG_ERR_ARG if more
 * functions reach one cell or element than the integration kernels hold. */
mlpg_status mlpg_integrate(mlpg_ctx *ctx);

/* Quadrature-outermost integration of every bilinear / linear form of the
 * SUPG weak transport equation (Alg. 1, Eq. weak-transport).  MLPG_ERR_STATE
 * unless integrated; MLPG_ERR_RK_SINGULAR, MLPG_ERR_ARG (too many functions
 * reach one element) or MLPG_ERR_GEOMETRY (a supported pair outside the overlap
 * pattern) from the device checks. */
mlpg_status mlpg_assemble(mlpg_ctx *ctx);

/* One backward-Euler step (Sec. 4.1) solved as in Sec. 4.2: first-flight
 * batched transport solves, GMRES (or source iteration, outer_method) on the
 * scalar-flux coefficients (Eq. krylov-operator) whose operator applies the
 * batched transport solve, angular recovery.  MLPG_MIXED wraps this in FP64
 * iterative refinement of the step with FP32 corrections.  dt = INFINITY
 * solves the steady problem.  Changing dt only re-forms the operators.
 * MLPG_ERR_NOT_CONVERGED on an FP64 iteration cap or when the refinement does
 * not converge in max_refine sweeps. */
mlpg_status mlpg_step(mlpg_ctx *ctx, double dt);

/* One backward-Euler step (as mlpg_step) of each of `count` independent
 * problems, run concurrently: the caller's thread steps ctxs[0] and one host
 * thread per further context steps the others, each on its own context
 * stream, so their kernels overlap on the device.  dt[i] is problem i's step.
 * The contexts must be distinct and must not share a stream (contexts created
 * with a NULL stream own one): otherwise MLPG_ERR_ARG before any step.
 * Returns MLPG_OK when every step succeeded, else the first failing status in
 * index order; each context's mlpg_last_error describes its own failure.
 * status[count] (may be NULL) receives every context's own status, so that a
 * caller can retire the failed problems and keep the others (whose steps are
 * done); on an argument error it is left unwritten.  The paper states the
 * problem for one point set; batching independent problems has no counterpart
 * there. */
mlpg_status mlpg_step_batch(mlpg_ctx *const *ctxs, const double *dt, int count, mlpg_status *status);

/* Scalar flux: kind 0 = point values phi_i = sum_j V_j U_j(x_i) Phi_j
 * (Eq. flux-expansion), kind 1 = coefficients Phi_i.  out[n], host; returns
 * when out is written.  MLPG_ERR_STATE before integrate, MLPG_ERR_ARG for
 * another kind. */
mlpg_status mlpg_scalar_flux(mlpg_ctx *ctx, double *out, int kind);

/* Same with a device pointer out[n]; the work is queued on the library stream
 * and the call returns without waiting (synchronise that stream before
 * reading out). */
mlpg_status mlpg_scalar_flux_dev(mlpg_ctx *ctx, double *out, int kind);

/* Angular flux coefficients Psi[n*m] ([i][m] layout), host: the state of the
 * time-dependent problem (Sec. 4.1), read back and restored for checkpoints
 * (a library service; the paper has no restart).  mlpg_set_state is
 * mlpg_set_initial with a non-NULL psi. */
mlpg_status mlpg_get_state(const mlpg_ctx *ctx, double *psi);
mlpg_status mlpg_set_state(mlpg_ctx *ctx, const double *psi);

/* Counters of this context (mlpg_stats); the iteration counts are those of
 * Sec. 5.3's outer and inner solves.  MLPG_ERR_ARG for NULL arguments. */
mlpg_status mlpg_get_stats(const mlpg_ctx *ctx, mlpg_stats *stats);

/* Enable device timing of the batched L-apply launches (CUDA events on the
 * library stream); the totals appear in mlpg_stats.spmm_ms.  A measurement
 * service with no paper counterpart. */
mlpg_status mlpg_enable_timing(mlpg_ctx *ctx, int on);

/* ---- stage outputs, for inspection and parity checks -------------------- */

/* Overlap pattern (Sec. 3.4): rowptr[n+1], col[nnz], columns ascending. */
mlpg_status mlpg_get_neighbors(const mlpg_ctx *ctx, int64_t *rowptr, int32_t *col);

/* Cell volumes V_i (Sec. 3.1), host out[n]. */
mlpg_status mlpg_get_volumes(const mlpg_ctx *ctx, double *out);

/* The integrated forms of Eq. weak-transport (Sec. 4.1, Alg. 1).  Number of
 * integrated matrices / vectors and their values in this order:
 *   matrices (nnz each): M0, Mt, Ms, G^a (dim), Gt^a (dim), Gs^a (dim),
 *                        K^ab (dim*dim, a-major), S_f (2*dim)
 *   vectors (n each):    Q0, Q^a (dim), B_f (2*dim)
 * with test function U_i (row) and trial function V_j U_j (column):
 *   M0 <U_i,V_jU_j>, Mt/Ms with sigma_t/sigma_s, G^a <d_a U_i, V_jU_j>,
 *   K^ab <d_a U_i, d_b V_jU_j>, S_f (U_i, V_jU_j) on face f, Q0 <U_i,q>,
 *   Q^a <d_a U_i, q>, B_f (U_i, 1) on face f.  Host out arrays
 * mats[n_matrices * nnz], vecs[n_vectors * n].  MLPG_ERR_STATE before
 * assemble. */
int mlpg_n_matrices(int dim);
int mlpg_n_vectors(int dim);
mlpg_status mlpg_get_forms(const mlpg_ctx *ctx, double *mats, double *vecs);

/* Batched transport operator (Sec. 4.2, operator L): Y[i][m] = (L_m X_m)_i
 * for all directions at once, for the 1/(c dt) of `dt`; X, Y device [n][m]
 * arrays of `precision` (MLPG_FP64: double, MLPG_MIXED: float), queued on the
 * library stream; X and Y must not overlap and must start on 16-byte
 * boundaries (the kernels move four floats or two doubles at a time).
 * MLPG_ERR_STATE before assemble, MLPG_ERR_ARG for another precision,
 * dt <= 0 or a misaligned or overlapping X or Y. */
mlpg_status mlpg_apply_L_dev(mlpg_ctx *ctx, double dt, int precision, const void *X, void *Y);

/* ---- allocation-free helper ----------------------------------------------- */

/* Largest n accepted by mlpg_overlap_counts_noalloc. */
#define MLPG_NOALLOC_MAX_POINTS 262144

/* Row sizes of the overlap pattern, counts[i] = #{j : |x_i - x_j| < R_i + R_j},
 * for callers that cannot allocate device memory when they need them: code
 * running while a stream is captured into a CUDA graph, code living inside a
 * device memory budget fixed at start-up, real-time loops that must not touch
 * the allocator.  With the counts such a caller can size its own buffers.
 * The paper has no counterpart of this call (it is a service of this library);
 * the counts equal the row lengths of the pattern mlpg_integrate builds.
 *   points[n*dim], kernel_extent[n]: device arrays (finite, extents > 0,
 *                                    points inside [lo, hi])
 *   lo[dim], hi[dim]:                host arrays, the box
 *   counts[n]:                       device output (int32)
 *   stream:                          cudaStream_t, NULL = legacy default stream
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.  The
 * scratch is one static device array of about 2.8 MB that every GPU loading
 * this library holds until the process exits; n > MLPG_NOALLOC_MAX_POINTS
 * returns MLPG_ERR_ARG, as do a non-finite or empty box.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture.  The kept address belongs to the device's
 * primary context: after cudaDeviceReset on that device it is stale and the
 * call must not be used again in that process.  All calls share the one array: calls
 * that overlap on the GPU (different streams, or host threads without
 * ordering) race and give wrong counts; order them on one stream.  Work is
 * queued on `stream` and the call returns without waiting. */
mlpg_status mlpg_overlap_counts_noalloc(int dim, int64_t n, const double *points,
                                        const double *kernel_extent, const double *lo,
                                        const double *hi, int32_t *counts, void *stream);

/* ---- direction shards ------------------------------------------------------ */

/* Sum across direction shards (Sec. 4.2: L^-1 is block-diagonal in angle, so
 * the directions of one problem can be split over several contexts, one per
 * GPU, each created with its own subset of ordinates and weights).  The shards
 * exchange only sums: the angular reduction D (an n-vector, once for the first
 * flight and once per outer iteration, plus the state's scalar flux) and the
 * two sums of squares of each FP64 step-residual norm.  The library calls
 * fn(buf, count, user) with a HOST buffer of `count` doubles holding this
 * shard's partial sums; fn must overwrite them with the sums over all shards
 * and return 0.  Every shard calls fn equally often with equal counts, in the
 * same order, because the outer solve is replicated on identical data.  A
 * nonzero return fails the call in progress with MLPG_ERR_ARG ("cross-shard
 * sum failed").  fn == NULL removes the callback (a single shard, the
 * default).  Valid in any state; the caller keeps `user` alive. */
typedef int (*mlpg_reduce_fn)(double *buf, int64_t count, void *user);
mlpg_status mlpg_set_reduce(mlpg_ctx *ctx, mlpg_reduce_fn fn, void *user);

/* Last error message of this context ("" when none; "null context" for NULL).
 * Valid until the next call on the context. */
const char *mlpg_last_error(const mlpg_ctx *ctx);

/* Waits for the context's stream, frees every device and pinned allocation and
 * the stream it owns (not a caller's stream); NULL is accepted.  The pointer
 * is invalid afterwards. */
void mlpg_destroy(mlpg_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MLPG_H */

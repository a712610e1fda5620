/*
 * ibem.h - C ABI of the GB300 isogeometric single-layer BEM library (libibem).
 *
 * The library applies the Galerkin single-layer operator of the Laplace or
 * Helmholtz equation on a multipatch surface, discretised by patchwise tensor
 * B-splines S_{p,m} and compressed by an interpolation-based fast multipole
 * method (Doelz, Harbrecht, Kurz, Schoeps, Wolf, "A fast isogeometric BEM for
 * the three dimensional Laplace- and Helmholtz problems", Secs. 2-4).
 *
 * Conventions (all entry points):
 *  - Ownership: the caller owns every pointer it passes; the library owns only
 *    the device buffers inside a handle and frees them in ibem_destroy.
 *  - Pointers named *_dev are device pointers (CUDA global memory of the device
 *    that was current at ibem_create); every other pointer is host memory.
 *  - Vectors with several right-hand sides are stored right-hand side by
 *    right-hand side: element (r, i) of an [nrhs][n] array is at r * n + i.
 *  - Complex values (Helmholtz) are interleaved (re, im) doubles, so a complex
 *    [nrhs][n] array holds 2 * nrhs * n doubles.
 *  - Dof order of S_{p,m}: dof(patch, j_u, j_v) = patch * n1^2 + j_v * n1 + j_u
 *    with n1 = 2^m + p (j_u counts B-splines along the first parameter).
 *  - All device work is enqueued on the stream given to ibem_create.  Calls
 *    return after enqueueing, except where a comment says they synchronise.
 *  - Errors are returned as ibem_status; no C++ exception crosses the ABI.  The
 *    text of the last error of a handle is available from ibem_last_error.
 *  - A handle must not be used from two host threads at the same time.
 */
#ifndef IBEM_H
#define IBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibem_handle ibem_handle;

typedef enum {
    IBEM_OK = 0,
    IBEM_ERR_ARG = 1,        /* invalid argument (null pointer, size, option) */
    IBEM_ERR_GEOMETRY = 2,   /* invalid patch description or mesh topology   */
    IBEM_ERR_CUDA = 3,       /* a CUDA call failed; see ibem_last_error       */
    IBEM_ERR_OOM = 4,        /* device or host allocation failed             */
    IBEM_ERR_NOCONV = 5,     /* iterative solver reached maxit                */
    IBEM_ERR_BREAKDOWN = 6,  /* solver breakdown (p^T A p <= 0, NaN, ...)     */
    IBEM_ERR_STATE = 7       /* call out of order (e.g. matvec before assemble) */
} ibem_status;

/* Patch kinds (Sec. 2.2, Eq. def::geom). */
enum {
    IBEM_PATCH_NURBS = 0,       /* rational tensor B-spline map F : [0,1]^2 -> R^3 */
    IBEM_PATCH_SPHERE_FACE = 1  /* analytic cube-sphere face: F = c0 + R c/|c|,
                                   c = n + (2u-1) t1 + (2v-1) t2 for face 0..5
                                   (+x, -x, +y, -y, +z, -z)                      */
};

/* One patch, host memory; copied by ibem_create.
 * NURBS: degrees deg_u, deg_v >= 1 (<= 7), ncp_u x ncp_v control points,
 * knots_u has ncp_u + deg_u + 1 entries (open, non-decreasing, from 0 to 1),
 * ctrl_xyz is [ncp_v][ncp_u][3], weights is [ncp_v][ncp_u] and positive.
 * SPHERE_FACE: face in 0..5, radius > 0, center.
 * perturbed != 0 (either kind): the patch map becomes F(f(u), f(v)) with the
 * piecewise-linear f of Sec. 5 (perturbed mappings): f(x) = x / 2 on [0, 0.3],
 * 1.75 x - 0.375 on (0.3, 0.7), (x + 1) / 2 on [0.7, 1].  Same surface, same
 * patch corners, a parametrisation with kinks at 0.3 and 0.7 (H^1, not H^2);
 * its derivatives carry the factors f'(u), f'(v). */
typedef struct {
    int kind;
    int deg_u, deg_v, ncp_u, ncp_v;
    const double *knots_u, *knots_v, *ctrl_xyz, *weights;
    int face;
    double radius;
    double center[3];
    int perturbed;
} ibem_patch;

enum { IBEM_LAPLACE = 0, IBEM_HELMHOLTZ = 1 };   /* Eqs. fundament1 / fundament2 */

/* Arithmetic of the operator application. */
enum {
    IBEM_FP64 = 0,  /* FP64-accurate near field and coupling                   */
    IBEM_FP32 = 1,  /* FP32 near blocks, coupling generated on the fly in FP32,
                       FP32 accumulation (inputs and outputs stay FP64).  With
                       16..256 right-hand sides (and q even, 2 q^2 <= 128 for
                       Helmholtz, q^2 <= 128 for Laplace) the coupling is contracted on the
                       tensor cores: K and the moments in BF16, FP32 accumulation */
    IBEM_BF16 = 2   /* network entries only (ibem_cnn_*): BF16 activations and
                       weights, FP32 accumulation                              */
};

/* Preconditioners of ibem_solve: point Jacobi on the diagonal of T A_near T^T,
 * or block Jacobi on its diagonal blocks; a block holds the dofs whose last
 * support element lies in one cluster of level max(0, m - 2). */
enum { IBEM_PRECOND_NONE = 0, IBEM_PRECOND_JACOBI = 1, IBEM_PRECOND_BLOCK_JACOBI = 2,
       IBEM_PRECOND_LEARNED = 3   /* block-Jacobi plus the correction of an attached
                                     network, flexible GMRES (Helmholtz only); see
                                     ibem_set_learned_preconditioner */ };

typedef struct {
    int kernel;          /* IBEM_LAPLACE or IBEM_HELMHOLTZ                          */
    double kappa;        /* wavenumber (Helmholtz)                                  */
    int p;               /* spline degree, 0..4                                    */
    int m;               /* refinement level, 0..10: 4^m elements per patch         */
    int q_cheb;          /* Chebyshev points per direction per cluster (2..12); 0 =
                            no compression: every element pair is near field        */
    double eta;          /* admissible iff eta * max(diam) < dist (eta = 1/mu, Def. 4.1) */
    int gauss_regular;   /* Gauss points per direction (1..40, default 8) of regular
                            pairs, of each sub-square of near-singular pairs, of the
                            right-hand side and of the potentials (Sec. 4 item 4:
                            orders up to 40).  Above what a CTA can hold as a kernel
                            matrix in shared memory (about 12 for Laplace, 10 for
                            Helmholtz at p = 2) the near field is formed by a
                            streaming kernel (same sums).                            */
    int gauss_singular;  /* Gauss points per variable, Duffy rules (1..12, default 8) */
    int fp64_coupling;   /* storage and arithmetic of the FP64 operator's coupling:
                            IBEM_COUPLING_DF (0, default) or IBEM_COUPLING_NATIVE (1) */
    int admissibility;   /* reading of Def. 4.1 (printed as max diam < mu dist with
                            0 < mu < 1, while the workloads give eta = 1.6):
                            IBEM_ADMISSIBLE_ETA_DIAM (0, default): admissible iff
                            eta * max(diam) < dist (eta = 1/mu);
                            IBEM_ADMISSIBLE_ETA_DIST (1): iff max(diam) < eta * dist */
    int fp32_coupling;   /* coupling of the FP32 operator with 16..256 right-hand
                            sides (tensor cores): IBEM_FP32_COUPLING_GENERATE (0,
                            default) generates K per application; IBEM_FP32_
                            COUPLING_STORE (1) stores it in BF16 at assembly when it
                            fits in half of the free device memory (Helmholtz,
                            q = 8: 16 KB per far block) and streams it */
    int gauss_grading;   /* Gauss order raised towards the singularity (Sec. 4
                            item 4: logarithmically, up to 40), 0..39; 0 = off.
                            A non-touching near pair whose bounding balls give
                            rho = dist / max(diam) takes
                              n = min(40, gauss_regular + gauss_grading * k),
                            k the least integer >= 0 with 2^k rho >= 3/4 (rho = 0:
                            n = 40): gauss_grading more points per direction for
                            every halving of the relative distance.  Subdivided
                            pairs use n on each sub-square pair.  Touching pairs
                            keep their Duffy rules (gauss_singular).  Pairs whose
                            n differs from gauss_regular are formed by the
                            streaming kernel with their own rule. */
} ibem_params;

enum { IBEM_ADMISSIBLE_ETA_DIAM = 0, IBEM_ADMISSIBLE_ETA_DIST = 1 };
enum { IBEM_FP32_COUPLING_GENERATE = 0, IBEM_FP32_COUPLING_STORE = 1 };

/* FP64 coupling variants.  GB300 executes FP64 FMA at 1/64 of the FP32 rate, so
 * by default the coupling matrices are stored as unevaluated float pairs
 * (hi + lo, 8 bytes per real entry, 16 per complex one) and applied with exact
 * FP32 products and compensated sums (about 48 significant bits, relative
 * error ~1e-14).  NATIVE: Laplace stores doubles and uses FP64 FMA; Helmholtz
 * generates the coupling on the fly in FP64 (also chosen automatically when the
 * stored complex matrices would exceed half of the free device memory).  All
 * variants reproduce the FP64 oracle to 1e-12. */
enum { IBEM_COUPLING_DF = 0, IBEM_COUPLING_NATIVE = 1, IBEM_COUPLING_NONE = 2, IBEM_COUPLING_GENERATE = 3,
       IBEM_COUPLING_FP32_ONLY = 4, IBEM_COUPLING_SLICED = 5 };
/* IBEM_COUPLING_NONE stores no FP64 coupling matrices (memory for large
 * batches): the FP32 operator is available; the FP64 operator of a Laplace
 * handle then returns IBEM_ERR_STATE, Helmholtz generates it on the fly.
 * IBEM_COUPLING_GENERATE (Helmholtz): nothing is stored; every application
 * generates each far block once in double-float arithmetic (kernel values to
 * about 1e-13 relative) and applies it to all right-hand sides of the call
 * (chunks of up to 64), so the cost of the generation is shared by them.  This
 * is also what a Helmholtz handle with IBEM_COUPLING_DF or NONE does when the
 * stored matrices would not fit, for q <= 8 and a phase kappa |x - y| below
 * 90 on every far block;
 * otherwise the generation runs in native FP64 per right-hand side.  A Laplace
 * handle treats GENERATE like IBEM_COUPLING_DF.
 * IBEM_COUPLING_SLICED (Helmholtz, q_cheb = 8): like GENERATE, but the
 * contraction runs on the tensor cores: each far block's double-float kernel
 * values and each cluster's moments are split into 6 signed integer digits
 * (|d| <= 128, weights 2^-7, 2^-15, ..., 2^-47) under a power-of-two scale
 * (per block, per moment column), the 21 digit-slice products of combined
 * weight down to 2^-54 are accumulated exactly in FP32 (integer partial sums
 * below 2^23) and recombined in double-float, so the result carries about 45
 * significant bits, like GENERATE within the 1e-12 parity tolerance.  Chunks
 * of 32 right-hand sides.  Other handles (or a phase kappa |x - y| of 90 or more)
 * take the GENERATE path; a Laplace handle treats SLICED like DF.
 * IBEM_COUPLING_FP32_ONLY (memory for large batches): the FP64 near blocks are
 * released at the end of ibem_assemble, after the FP32 copy, the Jacobi
 * diagonal and the block-Jacobi inverses are formed from them, and no FP64
 * coupling is stored; only the FP32 operator is available (the FP64 operator,
 * ibem_solve and the training entry points return IBEM_ERR_STATE). */

typedef struct {
    int64_t ndof;          /* dim S_{p,m} = n (2^m + p)^2                          */
    int64_t ndof_super;    /* dim S*_{p,m} = n (2^m (p+1))^2                       */
    int64_t n_elements;    /* n 4^m                                                */
    int64_t n_clusters;    /* n (4^{m+1} - 1) / 3                                  */
    int64_t n_quad_points; /* n_elements * gauss_regular^2                          */
    int64_t n_near;        /* near-field element pairs                              */
    int64_t n_far;         /* far-field cluster pairs (all levels)                  */
    int64_t n_near_singular[4]; /* near pairs by class: identical, edge, vertex, subdivided */
    int64_t bytes_near;    /* device bytes of the stored FP64 near blocks           */
    int64_t bytes_far;     /* device bytes of the stored FP64 coupling matrices     */
    int assembled;         /* 1 after ibem_assemble                                 */
    int max_gauss_order;   /* largest Gauss order of a non-touching near pair       */
    int64_t n_near_graded; /* near pairs whose order differs from gauss_regular     */
    int stored_ring_depth; /* ring stages of the stored BF16 coupling kernel, timed
                              on the first stored application (0: not yet)     */
} ibem_info;

typedef struct {
    int iterations;        /* Krylov iterations, summed over the right-hand sides  */
    int outer;             /* restarts / iterative-refinement sweeps               */
    double rel_residual;   /* max over right-hand sides of |b - A w| / |b| with the
                              FP64 operator, recomputed at the end                 */
    double seconds;        /* wall time of the call                                 */
    int steps;             /* operator applications of the Krylov iterations (one
                              application serves every column of a block)          */
} ibem_solve_info;

/* Build the discretisation: patches, knot vectors, cluster tree and block
 * cluster tree (admissibility, Def. 4.1), pair classes of the near field, the
 * Bezier extraction operator T (Sec. 4.3), geometry tables at Gauss and
 * interpolation points (Sec. 3.2).  `cuda_stream` is a cudaStream_t (NULL =
 * legacy default stream).  Synchronises.  On error *out is NULL. */
ibem_status ibem_create(const ibem_patch* patches, int npatch, const ibem_params* params,
                        void* cuda_stream, ibem_handle** out);

/* Free every device and host buffer of the handle.  NULL is accepted. */
ibem_status ibem_destroy(ibem_handle* h);

/* Sizes and counts (host call, no device work). */
ibem_status ibem_get_info(const ibem_handle* h, ibem_info* info);

/* Assemble the near field (Galerkin blocks of element pairs in the Bernstein
 * superspace, Gauss and Duffy rules, Sec. 4 item 4) and the FMM coupling
 * matrices K of every far block (Sec. 4.2).  Synchronises. */
ibem_status ibem_assemble(ibem_handle* h);

/* Physical Gauss points where the caller samples boundary data:
 * xyz_dev is [n_quad_points][3] doubles (element by element). */
ibem_status ibem_quad_points(const ibem_handle* h, double* xyz_dev);

/* Right-hand side b = T g*, b_i = int_Gamma g b_i (Sec. 3.2, Sec. 4.3):
 * g_dev is [nrhs][n_quad_points] samples of g at ibem_quad_points (complex for
 * Helmholtz), b_dev is [nrhs][ndof] (complex for Helmholtz). */
ibem_status ibem_rhs(ibem_handle* h, const double* g_dev, int nrhs, double* b_dev);

/* y = T A T^T x (Sec. 4.3): the FMM-compressed single-layer Galerkin matrix in
 * S_{p,m}.  x_dev, y_dev are [nrhs][ndof] (complex for Helmholtz); they must
 * not overlap.  precision is IBEM_FP64 or IBEM_FP32.  Requires ibem_assemble. */
ibem_status ibem_matvec(ibem_handle* h, const double* x_dev, double* y_dev, int nrhs,
                        int precision);

/* Same as ibem_matvec with x and y in HOST memory: copies in, applies, copies
 * out, synchronises.  For callers without device buffers. */
ibem_status ibem_matvec_host(ibem_handle* h, const double* x, double* y, int nrhs,
                             int precision);

/* Solve T A T^T w = b (Sec. 4 item 3): Jacobi-preconditioned conjugate
 * gradients (Laplace) or GMRES(100) (Helmholtz); flexible GMRES(100) with
 * IBEM_PRECOND_LEARNED.  Stops when |b - A w| / |b| <= rtol with A the FP64
 * operator, for every right-hand side.
 * nrhs = 1: precision IBEM_FP64 runs the solver on the FP64 operator;
 * IBEM_FP32 runs it on the FP32 operator and replaces the recursive residual
 * by the true FP64 residual b - A w whenever it has dropped 100-fold (CG,
 * reliable updates) or at every restart (GMRES); info->outer counts them.
 * maxit bounds the iterations.
 * nrhs > 1: all right-hand sides are solved together in lock step (each has
 * its own Krylov space and stopping test; one operator application per step
 * serves all of them, so the many-right-hand-side operators run inside the
 * solve).  Outer loop: the true FP64 residual of every column; converged
 * columns leave the block; the others take one GMRES(100) cycle (or one CG
 * run) on A d = r and x += d.  With IBEM_FP64 the inner solve aims at rtol;
 * with IBEM_FP32 it runs on the FP32 operator (tensor-core coupling from 16
 * columns on) to max(rtol |b|, 1e-3 |r|), so the outer loop is iterative
 * refinement with FP64 residuals.  maxit bounds the lock-step operator
 * applications (info->steps).
 * Synchronises; returns IBEM_ERR_NOCONV if maxit is reached. */
ibem_status ibem_solve(ibem_handle* h, const double* b_dev, double* w_dev, int nrhs,
                       double rtol, int maxit, int precond, int precision,
                       ibem_solve_info* info);

/* Potential u(x) = int_Gamma u*(x, y) w_h(y) dy (Eq. repform) at npts points
 * (pts_dev [npts][3]) by Gauss quadrature on every element; w_dev [nrhs][ndof],
 * u_dev [nrhs][npts] (complex for Helmholtz). */
ibem_status ibem_potential(ibem_handle* h, const double* w_dev, int nrhs,
                           const double* pts_dev, int64_t npts, double* u_dev);

/* The same potential with the far field interpolated (Sec. 4.2 applied to
 * Eq. repform).  Per point the cluster tree is walked from the patch roots: a
 * cluster tau with eta * diam(tau) < max(0, |x - c_tau| - r_tau) (the point as a
 * ball of radius 0 in Def. 4.1; c, r the cluster's bounding ball) contributes
 * sum_b u*(x, F(z_b)) k(z_b) x^_tau[b] from the density's forward moments
 * x^_tau (the q x q Chebyshev points z_b of the handle), an element that is
 * never admissible contributes its n x n Gauss sum as in ibem_potential, any
 * other cluster is split into its four children.  Same arguments, layouts and
 * units as ibem_potential; needs a compressed handle (q_cheb > 0; IBEM_ERR_ARG
 * otherwise), not the assembled operator.  The error against ibem_potential is
 * the interpolation error of the kernel on admissible clusters (it falls
 * geometrically in q).  Builds per-point interaction lists on the device, with
 * one host synchronisation to size them, and forms the moments of the clusters
 * the lists use only; temporary device memory (released on the stream): the
 * lists, the moments (8 q^2 bytes per used cluster and real density vector;
 * complex densities count twice), the split complex densities and, when some
 * element is near a point, the lifted densities (8 ndof_super bytes per real
 * vector).  The first call also builds the handle's 1D moment tables.  n_far_terms and
 * n_near_terms (may be null) receive the total number of (point, cluster) and
 * (point, element) terms.  A device-side overflow of the fixed traversal stack
 * (not reachable for m <= 10) records IBEM_DEVICE_OVERFLOW in the status word.
 * At most 2^31 - 1 points and 262,140 densities per call (IBEM_ERR_ARG). */
ibem_status ibem_potential_fmm(ibem_handle* h, const double* w_dev, int nrhs,
                               const double* pts_dev, int64_t npts, double* u_dev,
                               int64_t* n_far_terms, int64_t* n_near_terms);

/* Per-phase timing of operator applications (tracing).  Phases: 0 lift (T^T),
 * 1 upward pass (leaf moments, M2M), 2 far-field coupling, 3 downward pass
 * (L2L, back-projection), 4 near-field product, 5 restriction (T).  While
 * enabled, every ibem_matvec records a CUDA event pair around each phase on the
 * handle's stream.  `launches` counts the library's kernel launches of all
 * applications since the last read, enabled or not. */
typedef struct {
    int64_t applications;  /* operator applications recorded                    */
    int64_t launches;      /* kernels launched by operator applications         */
    double ms[6];          /* summed device time per phase                        */
} ibem_profile_data;

/* Enable (1) or disable (0) phase timing; clears the recorded data. */
ibem_status ibem_profile_enable(ibem_handle* h, int enable);

/* Synchronise the stream, return the sums since the last read/enable, clear. */
ibem_status ibem_profile_read(ibem_handle* h, ibem_profile_data* out);

/* Device-side waits.  Kernels that wait on asynchronous copies poll an
 * mbarrier at most `limit` times (default 2^26); a wait that runs out makes the
 * kernel record IBEM_DEVICE_TIMEOUT in the handle's status word, wait (bounded)
 * for its copies in flight and return without finishing its output, so the
 * CUDA context stays usable.  limit = 0 makes every such wait fail at once
 * (used to test the failure path). */
enum { IBEM_DEVICE_OK = 0, IBEM_DEVICE_TIMEOUT = 1,
       IBEM_DEVICE_OVERFLOW = 2   /* a fixed-size device work list would have
                                     overflowed; the kernel stopped that item */ };
ibem_status ibem_set_wait_limit(ibem_handle* h, long long limit);

/* Synchronise the stream, return the status word (IBEM_DEVICE_* bits) that the
 * kernels recorded since the last call, and clear it. */
ibem_status ibem_device_status(ibem_handle* h, int* status);

/* Potential evaluation that allocates no device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate at the
 * time they evaluate potentials: code recording a CUDA graph (cudaMalloc is
 * not permitted during stream capture), real-time loops that must not enter
 * the allocator, processes whose device memory is reserved up front by a pool
 * they do not control.  Same arguments, layouts and result as ibem_potential,
 * but the temporary data (the lifted density, 8 * ndof_super bytes rounded up
 * to 256, and the Gauss-point source table, 32 * n_quad_points bytes) lives in
 * one fixed array of IBEM_NOALLOC_SCRATCH_BYTES inside the library, held by
 * every GPU that loads libibem until the process exits.  A discretisation that
 * needs more returns IBEM_ERR_ARG with the required size in ibem_last_error.
 * The first call on a device looks the array up (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the one array:
 * calls whose GPU work can overlap (different streams or handles on one device
 * without ordering between them) race on it and must be serialised by the
 * caller.  The output u_dev is cleared by the call.  Laplace handles only
 * (a Helmholtz handle gets IBEM_ERR_ARG).  The looked-up address is kept for
 * the life of the process: after a device reset (cudaDeviceReset), which also
 * invalidates every handle on that device, do not call this entry point
 * again in the same process. */
#define IBEM_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
ibem_status ibem_potential_noalloc(ibem_handle* h, const double* w_dev, int nrhs,
                                   const double* pts_dev, int64_t npts, double* u_dev);

/* ---- Batches of uneven instances (no counterpart in the paper) ----
 * A batch applies the FP32 operator of many assembled handles (different
 * geometry, level, degree, kernel and number of right-hand sides) together:
 * every stage runs as one launch over all instances, the far-field coupling as
 * one persistent kernel balancing (instance, right-hand side, target cluster)
 * items through an atomic counter, and the application is captured once into a
 * CUDA graph and replayed.  The coupling kernel's CTA size is autotuned at
 * creation.  Handles must be assembled, with q_cheb in 2..8, on the current
 * device; they must outlive the batch.  nrhs[i] in 1..256.  `cuda_stream`
 * (NULL: the batch creates its own non-default stream). */
typedef struct ibem_batch ibem_batch;
ibem_status ibem_batch_create(ibem_handle* const* handles, int n, const int* nrhs, void* cuda_stream,
                              ibem_batch** out);
/* offsets[0..n]: instance i's input and output occupy doubles offsets[i] ..
 * offsets[i+1] of the concatenated arrays ([nrhs_i][ndof_i], complex interleaved). */
ibem_status ibem_batch_offsets(const ibem_batch* b, int64_t* offsets);
/* y = A x for every instance (FP32 operator, FP64 in and out), enqueued on the
 * batch stream as one graph launch (captured on first use for this (x, y) pair). */
ibem_status ibem_batch_matvec(ibem_batch* b, const double* x_dev, double* y_dev);
/* kernel launches in one application and the autotuned shape of the coupling
 * kernel: CTA size and right-hand sides per work item (4, 8 or 16).  Any
 * output may be null. */
ibem_status ibem_batch_info(const ibem_batch* b, int* launches_per_apply, int* coupling_threads,
                            int* coupling_rhs_tile);
/* Solve A x = b for every instance and right-hand side of the batch (Sec. 4
 * item 3, for many uneven problems at once): lock-step restarted GMRES(100)
 * over all columns of the concatenated arrays (layout of ibem_batch_offsets),
 * each column with its own Krylov space and stopping test, every step one
 * application of the batched FP32 operator; Laplace columns run the same
 * GMRES (real).  Outer loop: the residual b - A x with each instance's FP64
 * operator when every handle has one (the inner cycles then stop at
 * max(rtol |b|, 1e-3 |r|): iterative refinement to rtol in FP64), otherwise
 * with the batched FP32 operator (relative tolerances much below 1e-6 are then
 * out of reach).  precond: IBEM_PRECOND_NONE, JACOBI or BLOCK_JACOBI (each
 * instance's own).  maxit bounds the lock-step operator applications.
 * info->rel_residual is the largest relative residual of a column.  During
 * the call the instances' work runs on the batch stream; the handles must not
 * be used elsewhere meanwhile.  Synchronises; IBEM_ERR_NOCONV if maxit is
 * reached. */
ibem_status ibem_batch_solve(ibem_batch* b, const double* b_dev, double* x_dev, double rtol, int maxit, int precond,
                             ibem_solve_info* info);
ibem_status ibem_batch_destroy(ibem_batch* b);

/* Right-hand side of the field of point sources, g(x) = sum_j c_j u*(x, y_j)
 * (u* of the handle's kernel), as b = T g* with g*_i = int_Gamma g b*_i (Sec.
 * 3.2), the far field of every source interpolated (Sec. 4.2): per source the
 * cluster tree is walked as for a potential point (ibem_potential_fmm); on a
 * cluster sigma with eta * diam(sigma) < max(0, |y_j - c_sigma| - r_sigma) the
 * integrand k u*(F(.), y_j) is replaced by its q x q Chebyshev interpolant, so
 * b*_i gets sum_a c_j k(z_a) u*(F(z_a), y_j) int_sigma L_a b*_i; an element
 * that is never admissible takes the n x n Gauss rule of ibem_rhs.  The node
 * values of all clusters pass through the operator's downward transfers.  It
 * is the transpose of ibem_potential_fmm (u* is symmetric).
 * src_dev [nsrc][3] (sources, not on Gauss points of near elements),
 * charges_dev [nrhs][nsrc] (complex for Helmholtz), b_dev [nrhs][ndof]
 * (complex for Helmholtz).  Needs a compressed handle (q_cheb > 0;
 * IBEM_ERR_ARG otherwise), not the assembled operator.  One host
 * synchronisation: the per-source lists are copied to the host and turned into
 * lists per cluster and per element (sources ascending: repeated calls give
 * identical results).  Temporary device memory (released on the stream): the
 * lists, the node values (8 q^2 bytes per cluster and real vector; complex
 * counts twice) and the superspace vectors (8 ndof_super bytes per real
 * vector).  n_far_terms, n_near_terms (may be null): total (source, cluster)
 * and (source, element) terms.  At most 2^31 - 1 sources and 32,767 charge
 * vectors (IBEM_ERR_ARG).  nsrc = 0 gives b = 0. */
ibem_status ibem_rhs_sources(ibem_handle* h, const double* src_dev, const double* charges_dev, int nrhs,
                             int64_t nsrc, double* b_dev, int64_t* n_far_terms, int64_t* n_near_terms);

/* Switch the coupling of the FP32 tensor-core operator of an assembled handle
 * (see ibem_params.fp32_coupling): IBEM_FP32_COUPLING_STORE generates the BF16
 * blocks [Kr; Ki] of every far block once (16 KB each at q = 8) and streams
 * them in every later application; IBEM_FP32_COUPLING_GENERATE releases them.
 * STORE needs a Helmholtz handle with q_cheb = 8 (IBEM_ERR_ARG otherwise) and
 * returns IBEM_ERR_OOM, keeping the generating path, when the blocks exceed
 * half of the free device memory.  Synchronises; not concurrently with an
 * application on the handle.  IBEM_ERR_STATE before ibem_assemble. */
ibem_status ibem_set_fp32_coupling(ibem_handle* h, int mode);

/* Host-only: build the block cluster tree without a GPU and return its lists.
 * Call once with null arrays to get the counts.  near: [n_near][8] int32 =
 * (patch_t, ix_t, iy_t, patch_s, ix_s, iy_s, class, orientation) with class
 * 0 identical, 1 common edge, 2 common vertex, 3 subdivided, 4 regular and
 * orientation = 8 * k_target + k_source, k indexing the symmetries of the unit
 * square in the order (s,t), (1-t,s), (1-s,1-t), (t,1-s), (t,s), (1-s,t),
 * (1-t,1-s), (s,1-t).  far: [n_far][8] int32 = (patch, level, ix, iy)
 * of the target cluster then of the source cluster.  Lists are sorted. */
ibem_status ibem_block_tree(const ibem_patch* patches, int npatch, const ibem_params* params,
                            int64_t* n_near, int32_t* near, int64_t* n_far, int32_t* far);

/* Host-only: the Gauss order per direction of every near pair, in the order of
 * ibem_block_tree's near list: gauss_singular for touching pairs, the graded
 * order (see gauss_grading) for the others.  order: [n_near] int32, or null to
 * get the count only.  Errors as ibem_block_tree. */
ibem_status ibem_near_orders(const ibem_patch* patches, int npatch, const ibem_params* params, int64_t* n_near,
                             int32_t* order);

/* ---------------------------------------------------------------------------
 * Learned right preconditioner.  The paper has no counterpart (it preconditions
 * with Jacobi, Sec. 4 item 3); this is an addition of the library.
 *
 * Images: a complex vector of S_{p,m} is, patch by patch, an image of two
 * channels (real, imaginary part) and n1 x n1 pixels, pixel (j_v, j_u) of patch
 * k holding dof k * n1^2 + j_v * n1 + j_u.  Image arrays are FP32 device
 * memory [B][2][H][W].
 *
 * Network: four 3 x 3 convolutions with zero padding, channels
 * 2 -> C -> C -> C -> 2, ReLU after the first three.  Parameters are FP32,
 * flat, layer by layer: W[cout][cin][3][3] then bias[cout].  Loss of a batch of
 * B images: (1 / 2B) sum (net(in) - target)^2.  Optimiser: Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8, bias-corrected).
 *
 * Preconditioner: with s = B^-1 v the block-Jacobi vector and
 * sigma = |s| / sqrt(2 ndof), z = s + sigma * net(s / sigma) (network in BF16).
 * ibem_solve with IBEM_PRECOND_LEARNED runs flexible GMRES(100) with it.
 *
 * A network object is tied to the device current at creation and to the
 * stream given there (the preconditioner runs on the handle's stream).  It may
 * be attached to several handles; it must outlive them or be detached first.
 * --------------------------------------------------------------------------- */
typedef struct ibem_cnn ibem_cnn;

/* augmentation flags of ibem_cnn_train */
enum { IBEM_AUGMENT_PHASE = 1,      /* multiply input and target by e^{i theta}  */
       IBEM_AUGMENT_DIHEDRAL = 2 }; /* same symmetry of the square on both (H == W) */

/* New network with `channels` hidden channels (1..32), He-initialised from
 * `seed` (last layer scaled by 1/4, zero biases).  Synchronises. */
ibem_status ibem_cnn_create(int channels, unsigned long long seed, void* cuda_stream, ibem_cnn** out);
ibem_status ibem_cnn_destroy(ibem_cnn* cnn);

/* Parameter count into *count (if not null); copies the parameters to
 * get_host (if not null) after loading set_host (if not null; this also
 * resets the Adam state).  Synchronises. */
ibem_status ibem_cnn_params(ibem_cnn* cnn, float* get_host, const float* set_host, size_t* count);

/* out_dev = net(in_dev) for B images of H x W; precision IBEM_FP32 or
 * IBEM_BF16.  In BF16 with C = 32 all four layers run on the tensor cores
 * (tcgen05, BF16 operands, FP32 accumulation).  Enqueues only. */
ibem_status ibem_cnn_forward(ibem_cnn* cnn, const float* in_dev, int B, int H, int W, float* out_dev,
                             int precision);

/* Loss and its gradient with respect to the parameters (grad_host, FP32, the
 * parameter layout; loss in *loss), forward and backward in `precision`.
 * Either output may be null.  Synchronises. */
ibem_status ibem_cnn_gradients(ibem_cnn* cnn, const float* in_dev, const float* target_dev, int B, int H,
                               int W, int precision, float* grad_host, double* loss);

/* One Adam step with learning rate lr on one batch; the loss before the step in
 * *loss (synchronises if loss is not null). */
ibem_status ibem_cnn_train_step(ibem_cnn* cnn, const float* in_dev, const float* target_dev, int B, int H,
                                int W, float lr, int precision, double* loss);

/* Minibatch training in BF16: `epochs` passes over n_images (input, target)
 * images in a seeded random order, `batch` images per Adam step, with the
 * augmentations of `augment`.  *last_epoch_loss = mean over the images of the
 * last epoch of (1/2) |net(in) - target|^2.  Synchronises. */
ibem_status ibem_cnn_train(ibem_cnn* cnn, const float* in_dev, const float* target_dev, int n_images, int H,
                           int W, int batch, int epochs, float lr, unsigned long long seed, int augment,
                           double* last_epoch_loss);

/* Status word of the network's own device waits (bounded waits of the
 * tensor-core layers in ibem_cnn_forward), then cleared: 0 or
 * IBEM_DEVICE_TIMEOUT.  Synchronises.  Inside the preconditioner the handle's
 * status word (ibem_device_status) is used instead. */
ibem_status ibem_cnn_device_status(ibem_cnn* cnn, int* status);

/* Kernel launches of the network since the last call (then reset). */
ibem_status ibem_cnn_launches(ibem_cnn* cnn, int64_t* launches);

/* Coarse-grid variant of the preconditioner (factor f, 1..64; 1 = the fine
 * grid, the default): the network sees each patch image averaged over blocks
 * of f x f pixels (ragged blocks at the far edge average the pixels they hold)
 * and its correction is spread back over the blocks (piecewise constant):
 * z = s + sigma P net(R(s / sigma)); with f = 2^(m - l) it always sees the
 * level-l grid of a level-m discretisation.  Applies to the preconditioner and
 * to the residual-norm objective (ibem_cnn_operator_gradients,
 * ibem_cnn_train_operator), whose gradient passes through P^T (block sums). */
ibem_status ibem_cnn_set_coarsening(ibem_cnn* cnn, int factor);

/* Attach (or with NULL detach) a network as the learned preconditioner of a
 * Helmholtz handle.  The handle does not own it. */
ibem_status ibem_set_learned_preconditioner(ibem_handle* h, ibem_cnn* cnn);

/* z_dev = the learned preconditioner applied to v_dev (complex [ndof]; must
 * not overlap).  Requires ibem_assemble and an attached network. */
ibem_status ibem_learned_apply(ibem_handle* h, const double* v_dev, double* z_dev);

/* Residual/error training pairs from the plain solver: for every right-hand
 * side (b_dev, complex [nrhs][ndof]) block-Jacobi GMRES on the FP64 operator
 * runs to rtol; after every `stride`-th step of its first cycle (at most
 * max_pairs per right-hand side) the iterate x_k and its residual
 * r_k = b - A x_k (from the Arnoldi relation) are kept, and with x* the final
 * solution, e_k = x* - x_k, s_k = B^-1 r_k, sigma = |s_k| / sqrt(2 ndof) the
 * pair is written as images: in = s_k / sigma, target = (e_k - s_k) / sigma.
 * in_img_dev and tgt_img_dev hold nrhs * max_pairs * npatch images of
 * n1 x n1; pair n occupies images n * npatch ... (n + 1) * npatch - 1.
 * *n_pairs = pairs written.  Synchronises.  Returns IBEM_ERR_NOCONV (pairs
 * kept) if a solve did not reach rtol. */
ibem_status ibem_solver_pairs(ibem_handle* h, const double* b_dev, int nrhs, double rtol, int maxit,
                              int stride, int max_pairs, float* in_img_dev, float* tgt_img_dev,
                              int* n_pairs, ibem_solve_info* info);

/* Unit-norm residuals of the plain solver: for every right-hand side
 * block-Jacobi GMRES on the FP64 operator runs to rtol, and after every
 * `stride`-th step of its first cycle (at most max_vecs per right-hand side)
 * r_k / |r_k| (r_k = b - A x_k from the Arnoldi relation) is written to
 * r_out_dev (complex [nrhs * max_vecs][ndof]); *n_out = vectors written.
 * Synchronises.  IBEM_ERR_NOCONV (vectors kept) if a solve missed rtol. */
ibem_status ibem_solver_residuals(ibem_handle* h, const double* b_dev, int nrhs, double rtol, int maxit,
                                  int stride, int max_vecs, double* r_out_dev, int* n_out,
                                  ibem_solve_info* info);

/* Residual-norm objective of the learned preconditioner on unit-norm residuals
 * r_j (complex [n][ndof], n <= 256) of a Helmholtz handle:
 *   L = 1/(2n) sum_j |A z_j - r_j|^2,  z_j = s_j + sigma_j net(s_j / sigma_j),
 * s_j = B^-1 r_j.  Since A e_j = r_j this is the error z_j - e_j of the
 * residual/error pair measured in the norm |A .|.  The gradient passes through
 * A^H = conj(A conj(.)) (the Galerkin matrix is complex symmetric).
 * precision (network): IBEM_FP32 or IBEM_BF16; op_precision (operator):
 * IBEM_FP64 or IBEM_FP32.  grad_host / loss may be null.  Synchronises. */
ibem_status ibem_cnn_operator_gradients(ibem_handle* h, ibem_cnn* cnn, const double* r_dev, int n,
                                        int precision, int op_precision, float* grad_host, double* loss);

/* Adam training on that objective: `epochs` passes over the n residuals in a
 * seeded random order, minibatches of `batch` (<= 256) vectors, optional random
 * phase (IBEM_AUGMENT_PHASE), network in BF16, operator in op_precision.
 * *last_epoch_loss = mean over the vectors of the last epoch of
 * (1/2) |A z - r|^2.  Synchronises. */
ibem_status ibem_cnn_train_operator(ibem_handle* h, ibem_cnn* cnn, const double* r_dev, int n, int batch,
                                    int epochs, float lr, unsigned long long seed, int augment,
                                    int op_precision, double* last_epoch_loss);

/* Text of the last error recorded on the handle ("" if none).  NULL handle:
 * the last error of ibem_create / ibem_block_tree in this thread. */
const char* ibem_last_error(const ibem_handle* h);

/* Static name of a status code. */
const char* ibem_status_string(ibem_status s);

#ifdef __cplusplus
}
#endif

#endif /* IBEM_H */

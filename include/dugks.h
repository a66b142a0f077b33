/*
 * dugks.h -- C ABI of the GB300 DUGKS library: the discrete unified gas
 * kinetic scheme time step for the two-dimensional nonlinear
 * convection-diffusion equation (NCDE)
 *
 *     d_t phi + div B(phi) = div( alpha div D(phi) )                  (Eq. 2.1, F = 0)
 *
 * on a rectilinear (uniform or stretched) mesh with the D2Q9 velocity set
 * (Eq. 2.5), following Section 2 of arXiv:1906.11036.
 *
 * Conventions for every entry point:
 *   - No C++ exception crosses this boundary; every call returns a
 *     dugks_status.  CUDA failures map to DUGKS_ERR_CUDA and the CUDA error
 *     text is kept for dugks_last_error().
 *   - "device pointer" arguments must be device (or managed) memory of the
 *     GPU the context was created on, owned by the caller, aligned to the
 *     element size; "host pointer" arguments are ordinary (pageable or
 *     pinned) host memory owned by the caller.
 *   - All device work is enqueued on the context's CUDA stream (set at
 *     creation or by dugks_set_stream) and is asynchronous unless the entry
 *     point says that it synchronises.
 *   - Field layout: phi is [ny][nx] row-major (x fastest), contiguous.
 *     A distribution state is 9 planes [9][ny][nx], contiguous, velocity i
 *     ordered as in Eq. 2.5: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1)
 *     (-1,-1) (1,-1), times the lattice speed c.
 *   - Element type is float for precision 32 and double for precision 64,
 *     except where a signature says double.
 */
#ifndef DUGKS_H
#define DUGKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dugks_ctx dugks_ctx; /* opaque, library-owned */

typedef enum {
    DUGKS_OK = 0,
    DUGKS_ERR_ARG = 1,         /* null pointer, bad size, bad enum value */
    DUGKS_ERR_CONFIG = 2,      /* physically invalid setup (CFL >= 1, alpha <= 0, faces not increasing,
                                  negative initial equilibrium) */
    DUGKS_ERR_CUDA = 3,        /* a CUDA runtime or driver call failed */
    DUGKS_ERR_NONFINITE = 4,   /* NaN or Inf detected in phi */
    DUGKS_ERR_UNSUPPORTED = 5, /* valid request that the library does not implement */
    DUGKS_ERR_NOMEM = 6,       /* device or host allocation failed */
    DUGKS_ERR_TIMEOUT = 7      /* a bounded device-side wait expired; the step result is invalid */
} dugks_status;

enum { DUGKS_BC_PERIODIC = 0, DUGKS_BC_DIRICHLET = 1 };
enum { DUGKS_WALL_W = 0, DUGKS_WALL_E = 1, DUGKS_WALL_S = 2, DUGKS_WALL_N = 3 };
enum { DUGKS_D2Q9 = 9 };
enum { DUGKS_FP32 = 32, DUGKS_FP64 = 64 };
enum {
    DUGKS_KERNEL_AUTO = 0,  /* the fused streaming kernel */
    DUGKS_KERNEL_FUSED = 1, /* fused streaming kernel: TMA row pipeline, one read and one write of ftilde */
    DUGKS_KERNEL_NAIVE = 2  /* one thread per cell, everything recomputed from global memory (cross-check) */
};

/* Rectilinear mesh (Section 2: finite-volume cells V_j; Section 4, Example 4.3
 * for stretched meshes).  xf/yf are HOST arrays of nx+1 / ny+1 strictly
 * increasing face coordinates, copied at creation.  Cell centres are face
 * midpoints.  bc[] per wall W, E, S, N: DUGKS_BC_PERIODIC (must be set on both
 * walls of a direction) or DUGKS_BC_DIRICHLET with phi = bc_value[] on the
 * wall, imposed by a mirrored ghost cell with non-equilibrium extrapolation
 * (Section 4 opening names the scheme without defining it): the ghost sits at
 * the mirror image x_g = 2 x_w - x_1 of the first interior centre x_1, takes
 * phi_g = 2 phi_w - phi_1 and carries the interior cell's non-equilibrium part,
 * fbar+_g = feq(phi_g) + (fbar+_1 - feq(phi_1)); at the wall face the tangential
 * slope is the interior cell's alone, so corner ghosts are never used. */
typedef struct {
    int nx, ny;
    const double *xf;
    const double *yf;
    int bc[4];
    double bc_value[4];
} dugks_mesh;

/* Velocity set (Eq. 2.5): kind = DUGKS_D2Q9; c = lattice speed > 0, c_s^2 = c^2/3. */
typedef struct {
    int kind;
    double c;
} dugks_vset;

/* Coefficients (Eqs. 2.1, 2.3, Remark 3): B(phi) = u * b(phi),
 * D(phi) = d(phi) I, with b(phi) = sum_{k<nb} b[k] phi^k and
 * d(phi) = sum_{k<nd} d[k] phi^k; alpha > 0 is the diffusion coefficient and
 * fixes the relaxation time lambda = alpha / c_s^2 (Section 3).  The
 * auxiliary moment is C = u u * int_0^phi b'(s)^2 ds, or C = 0 if c_zero.
 * With d_tensor = 1, D is the symmetric tensor [[dxx, dxy], [dxy, dyy]](phi)
 * (each entry a polynomial with ndt <= 8 coefficients; d and nd are ignored),
 * as in Examples 4.4 (D = K phi / kappa) and 4.5 (D = diag(phi^nx, phi^ny)).
 * A zero-initialised tail keeps the isotropic D. */
typedef struct {
    double u[2];
    int nb;
    double b[8];
    double alpha;
    int nd;
    double d[8];
    int c_zero;
    int d_tensor;
    int ndt;
    double dxx[8], dxy[8], dyy[8];
} dugks_coef;

typedef struct {
    int precision; /* DUGKS_FP32 or DUGKS_FP64: storage and arithmetic type */
    int kernel;    /* DUGKS_KERNEL_* */
    void *stream;  /* cudaStream_t for all work; NULL = the legacy default stream */
    int device;    /* CUDA device ordinal; -1 = the current device */
} dugks_options;

typedef struct {
    int nx, ny, precision, kernel;
    long long pitch;        /* elements per row of one plane in the library's buffers */
    long long steps_done;   /* time steps taken since the last init/load */
    double dt, lambda, cfl; /* time step, relaxation time alpha/c_s^2, c dt / min cell width */
    int block_threads;      /* threads per block of the step kernel */
    int grid_blocks;        /* blocks per launch of the step kernel */
    long long state_bytes;  /* bytes of one ftilde buffer (two are held) */
    double time;            /* time of the current state (source terms only; see dugks_set_source) */
    int nsrc;               /* source terms set */
} dugks_info_t;

/* Validate a setup on the host only (no CUDA call).  Returns DUGKS_OK,
 * DUGKS_ERR_ARG (null pointers, nx or ny < 1, nb/nd outside 0..8, periodic set
 * on one wall of a direction only, unknown velocity set) or DUGKS_ERR_CONFIG
 * (non-finite values, faces not strictly increasing, c <= 0, alpha <= 0,
 * dt <= 0, or CFL = c dt / min cell width >= 1, the stability bound stated
 * in the opening of Section 4). */
dugks_status dugks_check_config(const dugks_mesh *mesh, const dugks_vset *vset,
                                const dugks_coef *coef, double dt);

/* Positivity of the equilibrium (Eq. 2.3) for phi in [phi_min, phi_max] (host
 * only, no CUDA call; 4097 samples of phi refined by golden-section search).
 * The equilibrium of Eq. 2.3 turns negative for large |B|/c (e.g. B =
 * (phi^2/2)(1, 1) with c = 1 and phi near 1: min f^eq = -0.24) and the scheme
 * is then not usable.  Rule: DUGKS_ERR_CONFIG if at some phi the smallest of
 * the nine f^eq_i(phi) is negative by more than 1e-3 of the largest |f^eq_i(phi)|
 * at the same phi (a marginal negativity is accepted: with D = phi^2 the
 * diagonal equilibria vanish at phi = 1/2 up to the small advective term).
 * *feq_min_out (nullable) receives the smallest f^eq_i(phi) itself.  Also
 * DUGKS_ERR_CONFIG for a non-finite coefficient, DUGKS_ERR_ARG for null
 * pointers, bad counts or phi_min > phi_max. */
dugks_status dugks_check_feq(const dugks_vset *vset, const dugks_coef *coef, double phi_min, double phi_max,
                             double *feq_min_out);

/* Create a context (Section 2, one time step of size dt per dugks_step).
 * Copies mesh and coefficients, precomputes per-row and per-column metrics
 * and the equilibrium polynomials, and allocates two ftilde buffers on the
 * device (library-owned; see dugks_info_t.state_bytes).  opts may be NULL
 * (FP32, fused kernel, default stream, current device).  On error *out is
 * set to NULL and nothing is leaked. */
dugks_status dugks_create(const dugks_mesh *mesh, const dugks_vset *vset, const dugks_coef *coef,
                          double dt, const dugks_options *opts, dugks_ctx **out);

/* Release the context and its device memory.  Synchronises the context's
 * stream first.  NULL is accepted and ignored. */
dugks_status dugks_destroy(dugks_ctx *ctx);

/* Initialise ftilde = feq(phi0) per cell (opening of Section 4), phi0 taken as
 * point values at cell centres.  phi0_dev: device pointer, [ny][nx], element
 * type of the context's precision.  Resets steps_done. */
dugks_status dugks_init_phi(dugks_ctx *ctx, const void *phi0_dev);

/* Same from a HOST array of doubles [ny][nx]; the copy goes through a
 * library-owned staging buffer on the context's stream.  Returns after the
 * host array may be reused (synchronises the stream). */
dugks_status dugks_init_phi_host(dugks_ctx *ctx, const double *phi0_host);

/* Advance n >= 0 time steps (Eq. 2.12 with the interface flux of Eqs.
 * 2.19-2.22 and Eq. 2.9), asynchronously on the context's stream.  One kernel
 * launch per step; the two ftilde buffers alternate. */
dugks_status dugks_step(dugks_ctx *ctx, long long n);

/* phi = sum_i ftilde_i (text after Eq. 2.13) into phi_dev_out (device,
 * [ny][nx], precision's element type; may be NULL) and, if mass_out is not
 * NULL, the mass M = sum |V_jk| phi_jk accumulated in double into *mass_out
 * (host).  With mass_out != NULL the call synchronises the stream and returns
 * DUGKS_ERR_NONFINITE if M is not finite. */
dugks_status dugks_get_phi(dugks_ctx *ctx, void *phi_dev_out, double *mass_out);

/* Same into a HOST array of doubles [ny][nx] (phi_host_out may be NULL);
 * synchronises the stream. */
dugks_status dugks_get_phi_host(dugks_ctx *ctx, double *phi_host_out, double *mass_out);

/* Copy the current ftilde state out to / in from a caller device buffer laid
 * out [9][ny][nx] (precision's element type).  Checkpoint and restart: a run
 * of n steps, save, load, m steps equals n + m steps bit for bit.  Loading
 * resets steps_done to 0. */
dugks_status dugks_save_state(dugks_ctx *ctx, void *f_dev_out);
dugks_status dugks_load_state(dugks_ctx *ctx, const void *f_dev_in);

/* Replace the stream used for subsequent work (NULL = legacy default). */
dugks_status dugks_set_stream(dugks_ctx *ctx, void *stream);

/* Synchronise the stream and report a pending device-side error flag
 * (DUGKS_ERR_TIMEOUT: a bounded wait expired; DUGKS_ERR_CONFIG: dugks_init_phi
 * met a negative equilibrium) or a CUDA error. */
dugks_status dugks_sync(dugks_ctx *ctx);

/* Failure-path check without a fault: launches one warp that waits at most
 * limit_us microseconds (1 ... 1000000) on an mbarrier that nothing completes,
 * the same bounded wait the step kernels use.  The wait expires and sets the
 * context's device error word, so the next dugks_sync returns
 * DUGKS_ERR_TIMEOUT (and keeps doing so: the context stays in the error state).
 * DUGKS_ERR_ARG for a null ctx or a limit outside the range. */
dugks_status dugks_wait_timeout_check(dugks_ctx *ctx, int limit_us);

/* Sizes and launch shape of a context. */
dugks_status dugks_info(const dugks_ctx *ctx, dugks_info_t *out);

/* ---- source terms ----------------------------------------------------------
 * Source F of Eq. 2.1 in the form F(x, t, phi) = sum_{k<nterms} exp(rate[k] t)
 * phi^power[k] S_k(x), S_k sampled at cell centres, with the source
 * distributions of Eq. 2.3: F_i = w_i F and, as Remark 3 reduces R_i for
 * B = u b(phi) and C = int B'B' dphi, R_i = w_i c_i.u b'(phi) F / c_s^2.
 * They enter the interface evolution of Eq. 2.18 and the update of Eq. 2.12;
 * the time derivatives there are the backward differences (S^n - S^{n-1})/dt
 * (S^{-1} = S^0 on the first step after dugks_set_source, dugks_init_phi or
 * dugks_load_state).
 *
 * fields_dev: device, [nterms][ny][nx] contiguous, precision's element type,
 * copied into library-owned memory (the caller may free it after the call
 * returns; the copy is ordered on the context's stream).  rate, power: host
 * arrays of nterms; 0 <= power[k] <= 15; nterms in 0..8 (0 removes the
 * source).  t0 is the time of the current state and of every later
 * dugks_init_phi; each step advances it by dt (dugks_info_t.time).
 * Errors: DUGKS_ERR_ARG (bad counts, null pointers, non-finite rates or t0),
 * DUGKS_ERR_UNSUPPORTED (C = 0, or the naive kernel), DUGKS_ERR_NOMEM.
 * The adjoint and batched entry points refuse a context with a source. */
dugks_status dugks_set_source(dugks_ctx *ctx, int nterms, const double *rate, const int *power,
                              const void *fields_dev, double t0);

/* ---- adjoint (gradients) -------------------------------------------------
 * Discrete adjoint of the step of Section 2 (reverse mode of Eqs. 2.9,
 * 2.12, 2.13, 2.19-2.22, 2.26 and of the mirrored NEE ghosts), for
 * gradients of a misfit J(phi^N) with respect to phi^0, alpha (alpha
 * enters through lambda = alpha / c_s^2, Section 3) and the velocity u of
 * the convection coefficients B = u b(phi), C = u u int b'^2 dphi (Remark 3),
 * which enter every f^eq of Eq. 2.3: cells, faces, ghosts and f^0.
 *
 * dugks_adjoint_step: lam = (d ftilde^{n+1} / d ftilde^n)^T mu at the forward
 * state f = ftilde^n, *dj_dalpha_dev += mu . d ftilde^{n+1} / d alpha and,
 * when dj_du_dev is not NULL, dj_du_dev[a] += mu . d ftilde^{n+1} / d u_a
 * (a = x, y).  f_dev, mu_dev, lam_dev: device, [9][ny][nx] contiguous,
 * precision's type (lam_dev must not alias f_dev or mu_dev); dj_dalpha_dev:
 * device double, or NULL (then only lam is returned); dj_du_dev: device, 2
 * doubles, or NULL (it needs dj_dalpha_dev); both accumulated in a fixed
 * order (deterministic).  Asynchronous. */
dugks_status dugks_adjoint_step(dugks_ctx *ctx, const void *f_dev, const void *mu_dev, void *lam_dev,
                                double *dj_dalpha_dev, double *dj_du_dev);

/* on = 1: every later initialisation tests the equilibrium of its phi0 by the
 * rule of dugks_check_feq.  dugks_init_phi_host applies it over the range of
 * its host phi0 and returns DUGKS_ERR_CONFIG before touching the state;
 * dugks_init_phi (device phi0) applies it per cell on the device, and the next
 * dugks_sync returns DUGKS_ERR_CONFIG if a cell failed.  Off by default: the
 * paper's own Example 4.1 takes phi (and with it f^eq) negative, which the
 * linear problem allows.  DUGKS_ERR_ARG for a null ctx or on outside 0..1. */
dugks_status dugks_set_feq_check(dugks_ctx *ctx, int on);

/* Which kernel runs an FP32 adjoint step (a cross-check hook; results agree to
 * FP32 rounding).  DUGKS_ADJ_AUTO (the default): the row-marching kernel
 * (periodic or Dirichlet walls) on grids with nx a multiple of 4 from 1 M
 * cells (1024^2), else the tiled kernel; DUGKS_ADJ_TILED: always the tiled kernel;
 * DUGKS_ADJ_ROWS: the row-marching kernel wherever it applies, whatever the
 * size.  DUGKS_ERR_ARG for a null ctx or an unknown value. */
enum { DUGKS_ADJ_AUTO = 0, DUGKS_ADJ_TILED = 1, DUGKS_ADJ_ROWS = 2 };
dugks_status dugks_set_adjoint_kernel(dugks_ctx *ctx, int kernel);

/* Gradient of J through nsteps steps from phi0: given grad_phiN = dJ/dphi^N
 * (device, [ny][nx]), writes dJ/dphi^0 into grad_phi0_dev (device [ny][nx]),
 * dJ/dalpha into *grad_alpha_out (host; may be NULL) and dJ/du into
 * grad_u_out[0..1] (host; may be NULL: the u-derivative is then not formed,
 * and the sweep reads less).  Runs the forward
 * sweep keeping one state every checkpoint_every steps, then for each segment
 * from the last recomputes its states and steps the adjoint back through it
 * (memory: ceil(nsteps/K) + K + 2 states of 9 nx ny elements in one workspace
 * that the context keeps for later calls, grown when a call needs more and
 * freed by dugks_destroy).  Synchronises the stream.  The context's own state
 * is left at an intermediate step: initialise it again before stepping. */
dugks_status dugks_adjoint(dugks_ctx *ctx, const void *phi0_dev, long long nsteps, int checkpoint_every,
                           const void *grad_phiN_dev, void *grad_phi0_dev, double *grad_alpha_out,
                           double *grad_u_out);

/* ---- batched instances ---------------------------------------------------
 * Many independent instances of the step of Section 2 (each with its own
 * mesh, coefficients and time step) advanced together: every time step is one
 * persistent launch whose warps take (instance, strip, row segment) tiles from
 * a global queue, largest instances first; runs of steps replay a captured
 * CUDA graph.  Single precision only (DUGKS_ERR_UNSUPPORTED otherwise), and
 * equilibrium polynomials of degree <= 3.  Instance i is addressed by its
 * index; its fields have the single-instance layouts. */
typedef struct dugks_batch dugks_batch;

/* Create n instances (arrays of n meshes, velocity sets, coefficients, time
 * steps).  opts may be NULL; opts->stream NULL makes the batch create its own
 * non-blocking stream.  Each instance is validated as by dugks_check_config. */
dugks_status dugks_batch_create(int n, const dugks_mesh *meshes, const dugks_vset *vsets, const dugks_coef *coefs,
                                const double *dts, const dugks_options *opts, dugks_batch **out);
dugks_status dugks_batch_destroy(dugks_batch *b);
/* ftilde = feq(phi0) for instance i (device [ny][nx] float); only before the first step. */
dugks_status dugks_batch_init_phi(dugks_batch *b, int i, const void *phi0_dev);
/* n time steps of every instance, asynchronous on the batch's stream. */
dugks_status dugks_batch_step(dugks_batch *b, long long n);
/* phi (and mass) of instance i, as dugks_get_phi. */
dugks_status dugks_batch_get_phi(dugks_batch *b, int i, void *phi_dev_out, double *mass_out);
/* ftilde of instance i into a device buffer [9][ny][nx], as dugks_save_state. */
dugks_status dugks_batch_save_state(dugks_batch *b, int i, void *f_dev_out);
/* Synchronise; DUGKS_ERR_TIMEOUT if a bounded device wait expired. */
dugks_status dugks_batch_sync(dugks_batch *b);
/* Autotuner: times steps_per_trial steps for each candidate tile height (rows
 * per tile, 8 ... 128), each without and with the split of every instance's
 * last rows (all but 0.8, 0.7 or 0.6 of them) into 8-row tiles queued after
 * all the others, on snapshots of the current states; keeps the fastest and
 * restores the states.
 * Outputs (nullable): the chosen rows per tile and milliseconds per step. */
dugks_status dugks_batch_autotune(dugks_batch *b, int steps_per_trial, int *best_rows_out, float *best_ms_out);
const char *dugks_batch_last_error(const dugks_batch *b);

/* ---- allocation-free variant -------------------------------------------
 * No counterpart in the paper: a convenience for callers that cannot
 * allocate device memory, for example a host application whose memory pool
 * already owns the GPU's free memory, or code that must not trigger the
 * device-wide synchronisation that cudaMalloc/cudaFree may imply.
 *
 * Computes the same phi = sum_i ftilde_i and mass M = sum |V_jk| phi_jk as
 * dugks_get_phi, without a context and without allocating anything: the
 * per-block partial sums live in a fixed array in the library's device
 * memory (DUGKS_NOALLOC_MAX_BLOCKS doubles = 512 KiB, present on every GPU
 * that loads the library until the process exits).
 *
 *   f_dev        device, [9][ny][nx] contiguous, float (precision 32) or double (64)
 *   dx_dev       device, nx doubles: cell widths in x; dy_dev: ny doubles in y
 *   phi_dev_out  device, [ny][nx] of the precision's type, or NULL
 *   mass_dev_out device, one double (written; not read)
 *   stream       cudaStream_t or NULL for the legacy default stream
 *
 * Asynchronous on `stream`.  Returns DUGKS_ERR_ARG for null pointers, a bad
 * precision or nx, ny < 1, and DUGKS_ERR_UNSUPPORTED when nx*ny exceeds
 * DUGKS_NOALLOC_MAX_CELLS (one partial sum per 256 cells), DUGKS_ERR_CUDA if
 * a launch of this call fails (an error left pending by earlier work of the
 * caller is neither cleared nor reported).  Every call looks up the array's
 * device address (cudaGetSymbolAddress, a host call) on the current device and
 * keeps nothing, so a call after cudaDeviceReset finds the new context's array;
 * make the first call on a device before any stream capture (that lookup may
 * load the library's device code).  All calls share the one array: calls that overlap on the GPU
 * (concurrent streams, or several host threads) race and must be serialised
 * by the caller.  Every partial sum is overwritten before it is read, so
 * nothing from an earlier call leaks into a later one. */
#define DUGKS_NOALLOC_MAX_BLOCKS 65536
#define DUGKS_NOALLOC_MAX_CELLS (256LL * DUGKS_NOALLOC_MAX_BLOCKS)
dugks_status dugks_phi_mass_noalloc(const void *f_dev, int precision, int nx, int ny, const double *dx_dev,
                                    const double *dy_dev, void *phi_dev_out, double *mass_dev_out, void *stream);

/* Static text for a status code; never NULL. */
const char *dugks_status_string(dugks_status s);

/* Text of the last error recorded on ctx (empty string if none; never NULL). */
const char *dugks_last_error(const dugks_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DUGKS_H */

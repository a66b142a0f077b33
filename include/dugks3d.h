/*
 * dugks3d.h -- C ABI of the three-dimensional DUGKS step (arXiv:1906.11036,
 * Section 2, with the D3Q15 velocity set of Eq. 2.28 or D3Q19 of Eq. 2.6).
 *
 * The step, the readings and the conventions are those of dugks.h, lifted to
 * three axes: a rectilinear mesh with faces xf, yf, zf; B(phi) = u b(phi) with
 * u in R^3; D(phi) = d(phi) I; C = u u int_0^phi b'(s)^2 ds (Remark 3) or 0.
 * At a face the reconstruction of Eqs. 2.19 and 2.20 uses the normal slope
 * between the two cells and, for each of the two tangential axes, the cell
 * central differences interpolated to the face (the interior cell's alone at
 * a Dirichlet wall); Dirichlet walls use the mirrored ghost with
 * non-equilibrium extrapolation.  All device arrays are contiguous,
 * distribution arrays [Q][nz][ny][nx] and scalar fields [nz][ny][nx], in the
 * context's precision (float for DUGKS_FP32, double for DUGKS_FP64).
 *
 * Status codes, precision constants and dugks_options come from dugks.h.  No
 * function takes ownership of a caller pointer; the context owns its buffers.
 */
#ifndef DUGKS3D_H
#define DUGKS3D_H

#include "dugks.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dugks_3d_ctx dugks_3d_ctx; /* opaque, library-owned */

enum { DUGKS_D3Q15 = 15, DUGKS_D3Q19 = 19 };
/* walls, in the order of dugks_3d_mesh.bc */
enum { DUGKS_3D_W = 0, DUGKS_3D_E = 1, DUGKS_3D_S = 2, DUGKS_3D_N = 3, DUGKS_3D_B = 4, DUGKS_3D_T = 5 };

/* Mesh: nx, ny, nz >= 1 cells; xf, yf, zf host arrays of nx+1, ny+1, nz+1
 * strictly increasing face coordinates (copied); bc[w] DUGKS_BC_PERIODIC or
 * DUGKS_BC_DIRICHLET for walls W, E (x), S, N (y), B, T (z), periodic on both
 * walls of an axis or on neither; bc_value[w] the Dirichlet value of phi. */
typedef struct {
    int nx, ny, nz;
    const double *xf;
    const double *yf;
    const double *zf;
    int bc[6];
    double bc_value[6];
} dugks_3d_mesh;

/* Velocity set: kind = DUGKS_D3Q15 (Eq. 2.28) or DUGKS_D3Q19 (Eq. 2.6); c the
 * lattice speed, c_s^2 = c^2/3. */
typedef struct {
    int kind;
    double c;
} dugks_3d_vset;

/* Coefficients (Eqs. 2.1, 2.3, Remark 3): B = u b(phi), D = d(phi) I with
 * b(phi) = sum_{k<nb} b[k] phi^k, d(phi) = sum_{k<nd} d[k] phi^k (nb, nd <= 8);
 * alpha > 0 fixes lambda = alpha / c_s^2; C = u u int_0^phi b'^2, or 0 if c_zero. */
typedef struct {
    double u[3];
    int nb;
    double b[8];
    double alpha;
    int nd;
    double d[8];
    int c_zero;
} dugks_3d_coef;

typedef struct {
    int nx, ny, nz, q, precision;
    long long steps_done;   /* steps since the last init/load */
    double dt, lambda, cfl; /* time step, alpha / c_s^2, c dt / min cell width */
    int block_threads;      /* threads per CTA of the step kernel */
    int grid[3];            /* CTAs: x strips, y row blocks, z segments */
    int zseg;               /* z-planes per CTA segment */
    long long state_bytes;  /* bytes of one ftilde buffer (two are held) */
} dugks_3d_info_t;

/* Host-only validation, as dugks_check_config: DUGKS_ERR_ARG for null
 * pointers, sizes < 1, nb/nd outside 0..8, an axis periodic on one wall only,
 * or an unknown velocity set; DUGKS_ERR_CONFIG for non-finite values, faces
 * not strictly increasing, c, alpha or dt <= 0, or CFL = c dt / min cell
 * width >= 1 (opening of Section 4). */
dugks_status dugks_3d_check_config(const dugks_3d_mesh *mesh, const dugks_3d_vset *vset,
                                   const dugks_3d_coef *coef, double dt);

/* Create a context (one time step of size dt per dugks_3d_step): copies the
 * mesh and coefficients, precomputes metrics and the equilibrium polynomials
 * of Eq. 2.3, allocates two ftilde buffers of Q nx ny nz elements.  opts may be
 * NULL (FP32, default stream, current device).  On error *out is NULL. */
dugks_status dugks_3d_create(const dugks_3d_mesh *mesh, const dugks_3d_vset *vset, const dugks_3d_coef *coef,
                             double dt, const dugks_options *opts, dugks_3d_ctx **out);

/* Release the context (synchronises its stream).  NULL is ignored. */
dugks_status dugks_3d_destroy(dugks_3d_ctx *ctx);

/* ftilde = feq(phi0) per cell (opening of Section 4); phi0_dev device
 * [nz][ny][nx] of the context's element type.  Resets steps_done. */
dugks_status dugks_3d_init_phi(dugks_3d_ctx *ctx, const void *phi0_dev);

/* n >= 0 time steps (Eq. 2.12 with the interface flux of Eqs. 2.19-2.22 and
 * Eq. 2.9), one kernel launch each, asynchronous on the context's stream. */
dugks_status dugks_3d_step(dugks_3d_ctx *ctx, long long n);

/* phi = sum_i ftilde_i into phi_dev_out (device [nz][ny][nx]; may be NULL) and,
 * if mass_out is not NULL, M = sum |V| phi accumulated in double into
 * *mass_out (host; synchronises, DUGKS_ERR_NONFINITE if M is not finite). */
dugks_status dugks_3d_get_phi(dugks_3d_ctx *ctx, void *phi_dev_out, double *mass_out);

/* Copy the state out to / in from a caller device buffer [Q][nz][ny][nx]
 * (asynchronous on the stream).  Loading resets steps_done. */
dugks_status dugks_3d_save_state(dugks_3d_ctx *ctx, void *f_dev_out);
dugks_status dugks_3d_load_state(dugks_3d_ctx *ctx, const void *f_dev_in);

/* Synchronise the stream; DUGKS_ERR_CUDA on a pending CUDA error. */
dugks_status dugks_3d_sync(dugks_3d_ctx *ctx);

dugks_status dugks_3d_info(const dugks_3d_ctx *ctx, dugks_3d_info_t *out);

/* Text of the last error recorded on ctx ("" if none). */
const char *dugks_3d_last_error(const dugks_3d_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* DUGKS3D_H */

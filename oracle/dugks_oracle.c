/*
 * dugks_oracle.c -- plain, slow, FP64 CPU implementation of the DUGKS time
 * step for the two-dimensional nonlinear convection-diffusion equation
 * (NCDE) with the D2Q9 velocity set, written from the paper's Section 2.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle: only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or helper with the CUDA library and
 * must never be reached from the product path.
 *
 * It follows the step summary at the end of Section 2 in the paper's order,
 * with explicit intermediate arrays:
 *   1. phi = sum_i ft_i                                   (text after Eq. 2.13)
 *   2. feq_i(phi)                                         (Eq. 2.3)
 *   3. fbp = fbar^+ (Eq. 2.21) and ftp = ftilde^+ (Eq. 2.13)
 *   4. ghost / halo cells (periodic wrap, or the Dirichlet reading below)
 *   5. x-faces: value and slopes (Eqs. 2.19, 2.20), fbar at x_b (Eq. 2.26,
 *      or Eq. 2.18 with sources), phi_b = sum_i fbar_i, feq(phi_b), f at the
 *      face (Eq. 2.22), flux (Eq. 2.9)
 *   6. y-faces likewise
 *   7. cell update ft^{n+1} = ftp - dt/|V| J (Eq. 2.12, with its source terms
 *      when a source F is given)
 *
 * Readings of points the paper leaves open (all shared with the CUDA path,
 * never its code):
 *   - Eq. 2.15 lost its f_i; read fbar = (2l+h)/(2l) f - h/(2l) feq.
 *   - Eq. 2.5 prints the diagonal weights with a garbled index; read
 *     w_5..w_8 = 1/36.
 *   - lambda = alpha / c_s^2 (Chapman-Enskog result, Section 3), h = dt/2.
 *   - The auxiliary moment C = u u * int_0^phi b'(s)^2 ds (Remark 3) for
 *     B = u b(phi), or C = 0 when requested; D = d(phi) I, or a symmetric
 *     tensor with polynomial entries [[dxx, dxy], [dxy, dyy]](phi).
 *   - Source F(x, t, phi) = sum_k exp(rate_k t) phi^pow_k S_k(x), S_k sampled
 *     at cell centres.  R_i follows Remark 3 (B = B(phi), C = int B'B' dphi):
 *     R_i = w_i c_i . B'(phi) F / c_s^2; sources are refused with C = 0.
 *   - The time derivatives of R_i and F_i in Eqs. 2.12 and 2.18 use the
 *     backward difference (S^n - S^{n-1}) / dt (the explicit form the text
 *     after Eq. 2.13 describes); on the first step S^{-1} = S^0.
 *   - At a Dirichlet wall the ghost cell's source distributions equal those
 *     of the interior cell next to it.
 *   - 2-D reconstruction at an x-face between cells j and j+1 (Eq. 2.20 is
 *     only given in 1-D): normal slope g_n = (P_{j+1}-P_j)/(x_{j+1}-x_j),
 *     value P_j + (x_b-x_j) g_n, tangential slope g_t = (1-w) G_j + w G_{j+1}
 *     with w = (x_b-x_j)/(x_{j+1}-x_j) and G the cell central difference
 *     (P_{k+1}-P_{k-1})/(y_{k+1}-y_{k-1}).  y-faces are symmetric.
 *   - Dirichlet walls (the paper cites a non-equilibrium extrapolation
 *     scheme without defining it): one ghost cell mirrored across the wall,
 *     x_g = 2 x_w - x_1, phi_g = 2 phi_w - phi_1, and
 *     fbp_g = feq(phi_g) + (fbp_1 - feq(phi_1)); at a wall face the
 *     tangential slope is the interior cell's G alone.
 *   - Periodic directions wrap the cell index and shift the coordinate by
 *     the domain length.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
#define BC_PERIODIC 0
#define BC_DIRICHLET 1
#define WALL_W 0
#define WALL_E 1
#define WALL_S 2
#define WALL_N 3

/* D2Q9 (Eq. 2.5): directions in units of c, and weights. */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

typedef struct {
    int nx, ny;
    const double *xf; /* nx+1 x-face coordinates, increasing */
    const double *yf; /* ny+1 y-face coordinates, increasing */
    int bc[4];        /* W, E, S, N: 0 periodic, 1 Dirichlet */
    double bc_value[4];
    double c;         /* lattice speed */
    double u[2];      /* B(phi) = u * b(phi) */
    int nb;
    double b[8];      /* b(phi) = sum_k b[k] phi^k */
    double alpha;     /* diffusion coefficient */
    int nd;
    double d[8];      /* D(phi) = d(phi) I, d(phi) = sum_k d[k] phi^k */
    int c_zero;       /* 1: C = 0 instead of u u int b'^2 */
    double dt;
    int d_tensor;     /* 1: D = [[dxx, dxy], [dxy, dyy]](phi) instead of d(phi) I */
    int ndt;          /* coefficients in each of dxx, dxy, dyy */
    double dxx[8], dxy[8], dyy[8];
    double t0;        /* time of the state given to oracle_step / oracle_run */
    int nsrc;         /* source terms: F = sum_k exp(rate_k t) phi^pow_k S_k(x) */
    double src_rate[8];
    int src_pow[8];
    const double *src_field; /* [nsrc][ny][nx], S_k at the cell centres */
} oracle_problem;

/* ------------------------------------------------------------------ */
/* Coefficient functions                                               */
/* ------------------------------------------------------------------ */

static double poly(int n, const double *a, double x) {
    double s = 0.0, p = 1.0;
    for (int k = 0; k < n; k++) {
        s += a[k] * p;
        p *= x;
    }
    return s;
}

/* int_0^phi b'(s)^2 ds with b'(s) = sum_k k b_k s^{k-1}:
 * b'^2 = sum_{k,l>=1} k l b_k b_l s^{k+l-2}, integrated term by term. */
static double aux_moment_scalar(const oracle_problem *p, double phi) {
    double s = 0.0;
    for (int k = 1; k < p->nb; k++)
        for (int l = 1; l < p->nb; l++) {
            int e = k + l - 1;
            s += (double)k * (double)l * p->b[k] * p->b[l] * pow(phi, (double)e) / (double)e;
        }
    return s;
}

/* Eq. 2.3: feq_i = w_i [phi + c_i.B/cs^2 + (cs^2 D + C - cs^2 phi I):(c_i c_i - cs^2 I)/(2 cs^4)] */
/* D(phi) as a 2x2 tensor: d(phi) I, or the polynomial tensor entries. */
static void diffusion_tensor(const oracle_problem *p, double phi, double D[2][2]) {
    if (p->d_tensor) {
        D[0][0] = poly(p->ndt, p->dxx, phi);
        D[0][1] = D[1][0] = poly(p->ndt, p->dxy, phi);
        D[1][1] = poly(p->ndt, p->dyy, phi);
    } else {
        const double dv = poly(p->nd, p->d, phi);
        D[0][0] = D[1][1] = dv;
        D[0][1] = D[1][0] = 0.0;
    }
}

/* derivative of a polynomial given by n coefficients */
static double poly_deriv(int n, const double *a, double x) {
    double s = 0.0, pw = 1.0;
    for (int k = 1; k < n; k++) { s += k * a[k] * pw; pw *= x; }
    return s;
}

void oracle_equilibrium(const oracle_problem *p, double phi, double *feq) {
    const double cs2 = p->c * p->c / 3.0;
    const double bv = poly(p->nb, p->b, phi);
    const double cv = p->c_zero ? 0.0 : aux_moment_scalar(p, phi);
    double B[2], T[2][2], D[2][2];
    diffusion_tensor(p, phi, D);
    for (int a = 0; a < 2; a++) B[a] = p->u[a] * bv;
    for (int a = 0; a < 2; a++)
        for (int e = 0; e < 2; e++) {
            double delta = (a == e) ? 1.0 : 0.0;
            T[a][e] = cs2 * D[a][e] + p->u[a] * p->u[e] * cv - cs2 * phi * delta;
        }
    for (int i = 0; i < Q; i++) {
        double ci[2] = {CX[i] * p->c, CY[i] * p->c};
        double cB = ci[0] * B[0] + ci[1] * B[1];
        double contr = 0.0;
        for (int a = 0; a < 2; a++)
            for (int e = 0; e < 2; e++) {
                double delta = (a == e) ? 1.0 : 0.0;
                contr += T[a][e] * (ci[a] * ci[e] - cs2 * delta);
            }
        feq[i] = WT[i] * (phi + cB / cs2 + contr / (2.0 * cs2 * cs2));
    }
}

/* d feq_i / d phi, term by term from Eq. 2.3: B' = u b', D' entrywise, C' = u u b'^2. */
void oracle_equilibrium_deriv(const oracle_problem *p, double phi, double *dfeq) {
    const double cs2 = p->c * p->c / 3.0;
    const double db = poly_deriv(p->nb, p->b, phi);
    double dD[2][2];
    if (p->d_tensor) {
        dD[0][0] = poly_deriv(p->ndt, p->dxx, phi);
        dD[0][1] = dD[1][0] = poly_deriv(p->ndt, p->dxy, phi);
        dD[1][1] = poly_deriv(p->ndt, p->dyy, phi);
    } else {
        dD[0][0] = dD[1][1] = poly_deriv(p->nd, p->d, phi);
        dD[0][1] = dD[1][0] = 0.0;
    }
    const double dc = p->c_zero ? 0.0 : db * db;
    double dB[2], dT[2][2];
    for (int a = 0; a < 2; a++) dB[a] = p->u[a] * db;
    for (int a = 0; a < 2; a++)
        for (int e = 0; e < 2; e++) {
            double delta = (a == e) ? 1.0 : 0.0;
            dT[a][e] = cs2 * dD[a][e] + p->u[a] * p->u[e] * dc - cs2 * delta;
        }
    for (int i = 0; i < Q; i++) {
        double ci[2] = {CX[i] * p->c, CY[i] * p->c};
        double contr = 0.0;
        for (int a = 0; a < 2; a++)
            for (int e = 0; e < 2; e++) {
                double delta = (a == e) ? 1.0 : 0.0;
                contr += dT[a][e] * (ci[a] * ci[e] - cs2 * delta);
            }
        dfeq[i] = WT[i] * (1.0 + (ci[0] * dB[0] + ci[1] * dB[1]) / cs2 + contr / (2.0 * cs2 * cs2));
    }
}

/* d feq_i / d u_a, a = x, y, for B = u b(phi) and C = u u int_0^phi b'^2 (Eq. 2.3, Remark 3):
 * c_i.B / c_s^2 gives w_i c_ia b / c_s^2 and C:(c_i c_i - c_s^2 I) / (2 c_s^4) gives
 * w_i Cint (c_ia (c_i.u) - c_s^2 u_a) / c_s^4 (the derivative of u u is symmetric). */
void oracle_equilibrium_du(const oracle_problem *p, double phi, double *dfx, double *dfy) {
    const double cs2 = p->c * p->c / 3.0;
    const double bv = poly(p->nb, p->b, phi);
    const double cv = p->c_zero ? 0.0 : aux_moment_scalar(p, phi);
    for (int i = 0; i < Q; i++) {
        const double ci[2] = {CX[i] * p->c, CY[i] * p->c};
        const double cu = ci[0] * p->u[0] + ci[1] * p->u[1];
        dfx[i] = WT[i] * (ci[0] * bv / cs2 + cv * (ci[0] * cu - cs2 * p->u[0]) / (cs2 * cs2));
        dfy[i] = WT[i] * (ci[1] * bv / cs2 + cv * (ci[1] * cu - cs2 * p->u[1]) / (cs2 * cs2));
    }
}

static double relax_time(const oracle_problem *p) { return p->alpha / (p->c * p->c / 3.0); }

/* Eqs. 2.21 and 2.13 for one cell: fbar^+ and ftilde^+ from ftilde and feq. */
void oracle_cell_transforms(const oracle_problem *p, const double *ft, const double *feq,
                            double *fbp, double *ftp) {
    const double lam = relax_time(p), dt = p->dt, h = 0.5 * p->dt;
    for (int i = 0; i < Q; i++) {
        fbp[i] = (2.0 * lam - h) / (2.0 * lam + dt) * ft[i] + 3.0 * h / (2.0 * lam + dt) * feq[i];
        ftp[i] = (2.0 * lam - dt) / (2.0 * lam + dt) * ft[i] + 2.0 * dt / (2.0 * lam + dt) * feq[i];
    }
}

/* Interface phi (text after Eq. 2.20) and Eq. 2.22 at one face: phi_b = sum fbar, then f = 2l/(2l+h) fbar + h/(2l+h) feq(phi_b). */
double oracle_face_original(const oracle_problem *p, const double *fbar, double *f) {
    const double lam = relax_time(p), h = 0.5 * p->dt;
    double phib = 0.0, feqb[Q];
    for (int i = 0; i < Q; i++) phib += fbar[i];
    oracle_equilibrium(p, phib, feqb);
    for (int i = 0; i < Q; i++)
        f[i] = 2.0 * lam / (2.0 * lam + h) * fbar[i] + h / (2.0 * lam + h) * feqb[i];
    return phib;
}

/* Eq. 2.1 source at cell c: F = sum_k exp(rate_k t) phi^pow_k S_k(x_c). */
double oracle_source(const oracle_problem *p, long c, double t, double phi) {
    const size_t n = (size_t)p->nx * p->ny;
    double s = 0.0;
    for (int k = 0; k < p->nsrc; k++)
        s += exp(p->src_rate[k] * t) * pow(phi, (double)p->src_pow[k]) * p->src_field[(size_t)k * n + (size_t)c];
    return s;
}

/* Eq. 2.3 source distributions at one cell: F_i = w_i F, and R_i = w_i c_i.(dB/dt + div C)/c_s^2,
 * which Remark 3 turns into R_i = w_i c_i.B'(phi) F / c_s^2 for B = u b(phi), C = int B'B' dphi. */
void oracle_source_distributions(const oracle_problem *p, double phi, double F, double *R, double *Fi) {
    const double cs2 = p->c * p->c / 3.0;
    const double db = poly_deriv(p->nb, p->b, phi);
    for (int i = 0; i < Q; i++) {
        const double ciBp = (CX[i] * p->c * p->u[0] + CY[i] * p->c * p->u[1]) * db;
        R[i] = WT[i] * ciBp * F / cs2;
        Fi[i] = WT[i] * F;
    }
}

/* ------------------------------------------------------------------ */
/* Initialisation and moments                                          */
/* ------------------------------------------------------------------ */

/* Section 4 opening: ft(x, 0) = feq(phi0) at each cell. f layout [Q][ny][nx]. */
void oracle_init(const oracle_problem *p, const double *phi0, double *f) {
    const size_t n = (size_t)p->nx * p->ny;
    for (size_t c = 0; c < n; c++) {
        double feq[Q];
        oracle_equilibrium(p, phi0[c], feq);
        for (int i = 0; i < Q; i++) f[i * n + c] = feq[i];
    }
}

void oracle_phi(const oracle_problem *p, const double *f, double *phi) {
    const size_t n = (size_t)p->nx * p->ny;
    for (size_t c = 0; c < n; c++) {
        double s = 0.0;
        for (int i = 0; i < Q; i++) s += f[i * n + c];
        phi[c] = s;
    }
}

/* M = sum_jk |V_jk| phi_jk, summed in a fixed serial order. */
double oracle_mass(const oracle_problem *p, const double *f) {
    const size_t n = (size_t)p->nx * p->ny;
    double m = 0.0;
    for (int k = 0; k < p->ny; k++)
        for (int j = 0; j < p->nx; j++) {
            size_t c = (size_t)k * p->nx + j;
            double s = 0.0;
            for (int i = 0; i < Q; i++) s += f[i * n + c];
            m += (p->xf[j + 1] - p->xf[j]) * (p->yf[k + 1] - p->yf[k]) * s;
        }
    return m;
}

/* ------------------------------------------------------------------ */
/* One time step                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    int nx, ny, ex, ey;   /* interior size and extended (1-cell halo) size */
    double *xc, *yc;      /* extended centre coordinates, index j+1 / k+1 */
    double *phi;          /* [ny][nx] */
    double *feq;          /* [Q][ny][nx] */
    double *fbp;          /* [Q][ey][ex] with halo */
    double *ftp;          /* [Q][ny][nx] */
    double *fx;           /* x-face flux c_ix f_i: [Q][ny][nx+1] */
    double *fy;           /* y-face flux c_iy f_i: [Q][ny+1][nx] */
    /* with sources: */
    double *sr, *sf;      /* R_i + h/2 dR_i/dt and F_i + h/2 dF_i/dt: [Q][ey][ex] with halo */
    double *rn, *fn;      /* R_i^n and F_i^n: [Q][ny][nx] */
    double *rp, *fp;      /* R_i^{n-1} and F_i^{n-1} (history kept by oracle_run) */
} workspace;

static int ws_alloc(workspace *w, const oracle_problem *p) {
    memset(w, 0, sizeof(*w));
    w->nx = p->nx;
    w->ny = p->ny;
    w->ex = p->nx + 2;
    w->ey = p->ny + 2;
    size_t n = (size_t)p->nx * p->ny, ne = (size_t)w->ex * w->ey;
    w->xc = malloc(sizeof(double) * w->ex);
    w->yc = malloc(sizeof(double) * w->ey);
    w->phi = malloc(sizeof(double) * n);
    w->feq = malloc(sizeof(double) * Q * n);
    w->fbp = malloc(sizeof(double) * Q * ne);
    w->ftp = malloc(sizeof(double) * Q * n);
    w->fx = malloc(sizeof(double) * Q * (size_t)p->ny * (p->nx + 1));
    w->fy = malloc(sizeof(double) * Q * (size_t)(p->ny + 1) * p->nx);
    if (!w->xc || !w->yc || !w->phi || !w->feq || !w->fbp || !w->ftp || !w->fx || !w->fy) return -1;
    if (p->nsrc > 0) {
        w->sr = malloc(sizeof(double) * Q * ne);
        w->sf = malloc(sizeof(double) * Q * ne);
        w->rn = malloc(sizeof(double) * Q * n);
        w->fn = malloc(sizeof(double) * Q * n);
        w->rp = malloc(sizeof(double) * Q * n);
        w->fp = malloc(sizeof(double) * Q * n);
        if (!w->sr || !w->sf || !w->rn || !w->fn || !w->rp || !w->fp) return -1;
    }
    /* extended centre coordinates: interior centres are face midpoints; ghost
     * centres are periodic images or mirror images across the wall. */
    const double Lx = p->xf[p->nx] - p->xf[0], Ly = p->yf[p->ny] - p->yf[0];
    for (int j = 0; j < p->nx; j++) w->xc[j + 1] = 0.5 * (p->xf[j] + p->xf[j + 1]);
    for (int k = 0; k < p->ny; k++) w->yc[k + 1] = 0.5 * (p->yf[k] + p->yf[k + 1]);
    if (p->bc[WALL_W] == BC_PERIODIC) {
        w->xc[0] = w->xc[p->nx] - Lx;
        w->xc[p->nx + 1] = w->xc[1] + Lx;
    } else {
        w->xc[0] = 2.0 * p->xf[0] - w->xc[1];
        w->xc[p->nx + 1] = 2.0 * p->xf[p->nx] - w->xc[p->nx];
    }
    if (p->bc[WALL_S] == BC_PERIODIC) {
        w->yc[0] = w->yc[p->ny] - Ly;
        w->yc[p->ny + 1] = w->yc[1] + Ly;
    } else {
        w->yc[0] = 2.0 * p->yf[0] - w->yc[1];
        w->yc[p->ny + 1] = 2.0 * p->yf[p->ny] - w->yc[p->ny];
    }
    return 0;
}

static void ws_free(workspace *w) {
    free(w->xc); free(w->yc); free(w->phi); free(w->feq);
    free(w->fbp); free(w->ftp); free(w->fx); free(w->fy);
    free(w->sr); free(w->sf); free(w->rn); free(w->fn); free(w->rp); free(w->fp);
}

/* element (i, k, j) of an extended [Q][ey][ex] array */
#define EXTA(w, X, i, k, j) ((X)[((size_t)(i) * (w)->ey + (size_t)(k)) * (w)->ex + (size_t)(j)])
#define EXT(w, i, k, j) EXTA(w, (w)->fbp, i, k, j)

/* NEE ghost of the reading above: interior cell (ji, ki) in extended
 * indices, ghost at (jg, kg), wall value phiw. */
static void nee_ghost(const oracle_problem *p, workspace *w, int jg, int kg, int ji, int ki, double phiw) {
    const size_t n = (size_t)p->nx * p->ny;
    size_t c = (size_t)(ki - 1) * p->nx + (size_t)(ji - 1);
    double phi1 = w->phi[c];
    double phig = 2.0 * phiw - phi1;
    double feqg[Q];
    oracle_equilibrium(p, phig, feqg);
    for (int i = 0; i < Q; i++)
        EXT(w, i, kg, jg) = feqg[i] + (EXT(w, i, ki, ji) - w->feq[i * n + c]);
}

static void fill_halo(const oracle_problem *p, workspace *w) {
    const int nx = p->nx, ny = p->ny;
    const int xper = p->bc[WALL_W] == BC_PERIODIC, yper = p->bc[WALL_S] == BC_PERIODIC;
    /* Dirichlet rows first (interior columns), then periodic x-wrap over all
     * rows including ghost rows (gives the corners when y is Dirichlet). */
    if (!yper)
        for (int j = 1; j <= nx; j++) {
            nee_ghost(p, w, j, 0, j, 1, p->bc_value[WALL_S]);
            nee_ghost(p, w, j, ny + 1, j, ny, p->bc_value[WALL_N]);
        }
    if (!xper)
        for (int k = 1; k <= ny; k++) {
            nee_ghost(p, w, 0, k, 1, k, p->bc_value[WALL_W]);
            nee_ghost(p, w, nx + 1, k, nx, k, p->bc_value[WALL_E]);
        }
    if (xper)
        for (int i = 0; i < Q; i++)
            for (int k = 0; k <= ny + 1; k++) {
                EXT(w, i, k, 0) = EXT(w, i, k, nx);
                EXT(w, i, k, nx + 1) = EXT(w, i, k, 1);
            }
    if (yper)
        for (int i = 0; i < Q; i++)
            for (int j = 0; j <= nx + 1; j++) {
                EXT(w, i, 0, j) = EXT(w, i, ny, j);
                EXT(w, i, ny + 1, j) = EXT(w, i, 1, j);
            }
    if (!xper && !yper) /* corners are never read with two walls: poison them */
        for (int i = 0; i < Q; i++) {
            EXT(w, i, 0, 0) = NAN;
            EXT(w, i, 0, nx + 1) = NAN;
            EXT(w, i, ny + 1, 0) = NAN;
            EXT(w, i, ny + 1, nx + 1) = NAN;
        }
}

/* Central difference of an extended array X in y at extended cell (j, k), velocity i. */
static double grad_y(const workspace *w, const double *X, int i, int k, int j) {
    return (EXTA(w, X, i, k + 1, j) - EXTA(w, X, i, k - 1, j)) / (w->yc[k + 1] - w->yc[k - 1]);
}
static double grad_x(const workspace *w, const double *X, int i, int k, int j) {
    return (EXTA(w, X, i, k, j + 1) - EXTA(w, X, i, k, j - 1)) / (w->xc[j + 1] - w->xc[j - 1]);
}

/* Eqs. 2.19 and 2.20 at x-face jf (between extended cells jf and jf+1) of row ke:
 * X(x_b - c_i h) = X(x_b) - h c_i . grad X(x_b), for the extended array X. */
static double recon_xface(const oracle_problem *p, const workspace *w, const double *X, int i, int ke, int jf) {
    const int jl = jf, jr = jf + 1, xper = p->bc[WALL_W] == BC_PERIODIC;
    const double h = 0.5 * p->dt, xb = p->xf[jf];
    const double dxc = w->xc[jr] - w->xc[jl];
    const double wgt = (xb - w->xc[jl]) / dxc;
    const double gn = (EXTA(w, X, i, ke, jr) - EXTA(w, X, i, ke, jl)) / dxc; /* Eq. 2.20 slope */
    const double val = EXTA(w, X, i, ke, jl) + (xb - w->xc[jl]) * gn;        /* Eq. 2.20 value */
    double gt;
    if (!xper && jf == 0)
        gt = grad_y(w, X, i, ke, jr); /* west wall: interior cell only */
    else if (!xper && jf == p->nx)
        gt = grad_y(w, X, i, ke, jl); /* east wall */
    else
        gt = (1.0 - wgt) * grad_y(w, X, i, ke, jl) + wgt * grad_y(w, X, i, ke, jr);
    return val - h * (CX[i] * p->c * gn + CY[i] * p->c * gt);
}

/* y-face kf (between extended rows kf and kf+1) of column je, likewise. */
static double recon_yface(const oracle_problem *p, const workspace *w, const double *X, int i, int kf, int je) {
    const int kl = kf, kr = kf + 1, yper = p->bc[WALL_S] == BC_PERIODIC;
    const double h = 0.5 * p->dt, yb = p->yf[kf];
    const double dyc = w->yc[kr] - w->yc[kl];
    const double wgt = (yb - w->yc[kl]) / dyc;
    const double gn = (EXTA(w, X, i, kr, je) - EXTA(w, X, i, kl, je)) / dyc;
    const double val = EXTA(w, X, i, kl, je) + (yb - w->yc[kl]) * gn;
    double gt;
    if (!yper && kf == 0)
        gt = grad_x(w, X, i, kr, je);
    else if (!yper && kf == p->ny)
        gt = grad_x(w, X, i, kl, je);
    else
        gt = (1.0 - wgt) * grad_x(w, X, i, kl, je) + wgt * grad_x(w, X, i, kr, je);
    return val - h * (CX[i] * p->c * gt + CY[i] * p->c * gn);
}

/* Halo of a source array: periodic images, or at a Dirichlet wall a copy of
 * the interior cell next to it (the reading in the header). */
static void fill_source_halo(const oracle_problem *p, workspace *w, double *X) {
    const int nx = p->nx, ny = p->ny;
    const int xper = p->bc[WALL_W] == BC_PERIODIC, yper = p->bc[WALL_S] == BC_PERIODIC;
    for (int i = 0; i < Q; i++) {
        for (int j = 1; j <= nx; j++) {
            EXTA(w, X, i, 0, j) = EXTA(w, X, i, yper ? ny : 1, j);
            EXTA(w, X, i, ny + 1, j) = EXTA(w, X, i, yper ? 1 : ny, j);
        }
        for (int k = 0; k <= ny + 1; k++) {
            EXTA(w, X, i, k, 0) = EXTA(w, X, i, k, xper ? nx : 1);
            EXTA(w, X, i, k, nx + 1) = EXTA(w, X, i, k, xper ? 1 : nx);
        }
        if (!xper && !yper) {
            EXTA(w, X, i, 0, 0) = NAN;
            EXTA(w, X, i, 0, nx + 1) = NAN;
            EXTA(w, X, i, ny + 1, 0) = NAN;
            EXTA(w, X, i, ny + 1, nx + 1) = NAN;
        }
    }
}

/* One step at time t.  With sources, R_prev / F_prev hold R_i^{n-1}, F_i^{n-1}
 * ([Q][ny][nx]; NULL on the first step) and R_i^n, F_i^n are left in w->rn, w->fn. */
static void step_ws(const oracle_problem *p, workspace *w, const double *f_in, double *f_out, double t,
                    const double *R_prev, const double *F_prev, int nthreads) {
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    const double h = 0.5 * p->dt, dt = p->dt;
    const double lam = relax_time(p);
    const int src = p->nsrc > 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif

    /* 1-3: phi, feq, fbar^+, ftilde^+ per cell; with sources also F, R_i, F_i (Eq. 2.3)
     * and their interface combinations S_i + h/2 dS_i/dt (Eq. 2.18) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < ny; k++)
        for (int j = 0; j < nx; j++) {
            size_t c = (size_t)k * nx + j;
            double ft[Q], feq[Q], fbp[Q], ftp[Q], phi = 0.0;
            for (int i = 0; i < Q; i++) { ft[i] = f_in[i * n + c]; phi += ft[i]; }
            oracle_equilibrium(p, phi, feq);
            oracle_cell_transforms(p, ft, feq, fbp, ftp);
            w->phi[c] = phi;
            for (int i = 0; i < Q; i++) {
                w->feq[i * n + c] = feq[i];
                w->ftp[i * n + c] = ftp[i];
                EXT(w, i, k + 1, j + 1) = fbp[i];
            }
            if (src) {
                double R[Q], Fi[Q];
                oracle_source_distributions(p, phi, oracle_source(p, (long)c, t, phi), R, Fi);
                for (int i = 0; i < Q; i++) {
                    const double Rp = R_prev ? R_prev[i * n + c] : R[i];
                    const double Fp = F_prev ? F_prev[i * n + c] : Fi[i];
                    w->rn[i * n + c] = R[i];
                    w->fn[i * n + c] = Fi[i];
                    EXTA(w, w->sr, i, k + 1, j + 1) = R[i] + 0.5 * h * (R[i] - Rp) / dt;
                    EXTA(w, w->sf, i, k + 1, j + 1) = Fi[i] + 0.5 * h * (Fi[i] - Fp) / dt;
                }
            }
        }
    /* 4: ghosts */
    fill_halo(p, w);
    if (src) {
        fill_source_halo(p, w, w->sr);
        fill_source_halo(p, w, w->sf);
    }
    /* weight of R in Eq. 2.18 */
    const double wr = 2.0 * lam * h / (2.0 * lam + h);

    /* 5: x-faces jf = 0..nx between extended cells jf (left) and jf+1 (right) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < ny; k++)
        for (int jf = 0; jf <= nx; jf++) {
            double fbar[Q], f[Q];
            for (int i = 0; i < Q; i++) {
                /* Eq. 2.19 + Eq. 2.26: fbar(x_b, t+h) = fbar^+(x_b) - h c_i . grad fbar^+(x_b) */
                fbar[i] = recon_xface(p, w, w->fbp, i, k + 1, jf);
                /* Eq. 2.18: + 2lh/(2l+h) [R_i + h/2 dR_i/dt] + h [F_i + h/2 dF_i/dt] at x_b - c_i h */
                if (src) fbar[i] += wr * recon_xface(p, w, w->sr, i, k + 1, jf) + h * recon_xface(p, w, w->sf, i, k + 1, jf);
            }
            oracle_face_original(p, fbar, f);
            for (int i = 0; i < Q; i++)
                w->fx[((size_t)i * ny + k) * (nx + 1) + jf] = CX[i] * p->c * f[i];
        }

    /* 6: y-faces kf = 0..ny */
#pragma omp parallel for schedule(static)
    for (int kf = 0; kf <= ny; kf++)
        for (int j = 0; j < nx; j++) {
            double fbar[Q], f[Q];
            for (int i = 0; i < Q; i++) {
                fbar[i] = recon_yface(p, w, w->fbp, i, kf, j + 1);
                if (src) fbar[i] += wr * recon_yface(p, w, w->sr, i, kf, j + 1) + h * recon_yface(p, w, w->sf, i, kf, j + 1);
            }
            oracle_face_original(p, fbar, f);
            for (int i = 0; i < Q; i++)
                w->fy[((size_t)i * (ny + 1) + kf) * nx + j] = CY[i] * p->c * f[i];
        }

    /* 7: cell update, Eq. 2.12 with J = sum over faces of (c_i . n) f_i |S|, plus
     * dt (S_i^n + dt/2 dS_i/dt) for S = R, F with dS/dt = (S^n - S^{n-1}) / dt */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < ny; k++)
        for (int j = 0; j < nx; j++) {
            size_t c = (size_t)k * nx + j;
            double dxj = p->xf[j + 1] - p->xf[j], dyk = p->yf[k + 1] - p->yf[k];
            double area = dxj * dyk;
            for (int i = 0; i < Q; i++) {
                double fe = w->fx[((size_t)i * ny + k) * (nx + 1) + j + 1];
                double fw = w->fx[((size_t)i * ny + k) * (nx + 1) + j];
                double fn = w->fy[((size_t)i * (ny + 1) + k + 1) * nx + j];
                double fs = w->fy[((size_t)i * (ny + 1) + k) * nx + j];
                double J = (fe - fw) * dyk + (fn - fs) * dxj;
                double v = w->ftp[i * n + c] - p->dt / area * J;
                if (src) {
                    const double R = w->rn[i * n + c], Fi = w->fn[i * n + c];
                    const double Rp = R_prev ? R_prev[i * n + c] : R;
                    const double Fp = F_prev ? F_prev[i * n + c] : Fi;
                    v += dt * (R + 0.5 * dt * (R - Rp) / dt) + dt * (Fi + 0.5 * dt * (Fi - Fp) / dt);
                }
                f_out[i * n + c] = v;
            }
        }
}

static int valid(const oracle_problem *p) {
    if (p->nx <= 0 || p->ny <= 0 || p->nb > 8 || p->nd > 8 || p->nb < 0 || p->nd < 0) return 0;
    if (p->d_tensor && (p->ndt < 0 || p->ndt > 8)) return 0;
    if (p->nsrc < 0 || p->nsrc > 8 || (p->nsrc > 0 && (!p->src_field || p->c_zero))) return 0;
    if ((p->bc[WALL_W] == BC_PERIODIC) != (p->bc[WALL_E] == BC_PERIODIC)) return 0;
    if ((p->bc[WALL_S] == BC_PERIODIC) != (p->bc[WALL_N] == BC_PERIODIC)) return 0;
    return p->alpha > 0.0 && p->c > 0.0 && p->dt > 0.0;
}

/* One step of the state at time p->t0 (with sources: the first step, no history). */
int oracle_step(const oracle_problem *p, const double *f_in, double *f_out, int nthreads) {
    workspace ws;
    if (!valid(p)) return -2;
    if (ws_alloc(&ws, p) != 0) { ws_free(&ws); return -1; }
    step_ws(p, &ws, f_in, f_out, p->t0, NULL, NULL, nthreads);
    ws_free(&ws);
    return 0;
}

/* One step with sources at time t, given R_i^{n-1}, F_i^{n-1} (NULL: first step);
 * R_i^n, F_i^n are written to R_out, F_out ([Q][ny][nx]). */
int oracle_step_src(const oracle_problem *p, const double *f_in, double *f_out, double t, const double *R_prev,
                    const double *F_prev, double *R_out, double *F_out, int nthreads) {
    workspace ws;
    if (!valid(p) || p->nsrc <= 0) return -2;
    if (ws_alloc(&ws, p) != 0) { ws_free(&ws); return -1; }
    step_ws(p, &ws, f_in, f_out, t, R_prev, F_prev, nthreads);
    const size_t sz = sizeof(double) * Q * (size_t)p->nx * p->ny;
    memcpy(R_out, ws.rn, sz);
    memcpy(F_out, ws.fn, sz);
    ws_free(&ws);
    return 0;
}

/* n steps in place on f from time p->t0 (ping-pong through a scratch copy);
 * with sources the R, F history starts at the first step. */
int oracle_run(const oracle_problem *p, double *f, long nsteps, int nthreads) {
    const size_t sz = sizeof(double) * Q * (size_t)p->nx * p->ny;
    workspace ws;
    if (!valid(p)) return -2;
    double *tmp = malloc(sz);
    if (!tmp || ws_alloc(&ws, p) != 0) { free(tmp); ws_free(&ws); return -1; }
    for (long s = 0; s < nsteps; s++) {
        const int hist = p->nsrc > 0 && s > 0;
        step_ws(p, &ws, f, tmp, p->t0 + (double)s * p->dt, hist ? ws.rp : NULL, hist ? ws.fp : NULL, nthreads);
        memcpy(f, tmp, sz);
        if (p->nsrc > 0) {
            memcpy(ws.rp, ws.rn, sz);
            memcpy(ws.fp, ws.fn, sz);
        }
    }
    ws_free(&ws);
    free(tmp);
    return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Adjoint of one time step (reverse mode of oracle_step)              */
/* ------------------------------------------------------------------ */
/*
 * Given f = ftilde^n and mu = dJ/d ftilde^{n+1}, returns lam = dJ/d ftilde^n
 * = (d step / d f)^T mu, and adds to *dj_dalpha the explicit dependence of
 * the step on alpha (through lambda = alpha / c_s^2 in the weights of Eqs.
 * 2.13, 2.21 and 2.22) contracted with mu, and to dj_du[0..1] (nullable) the
 * explicit dependence on u of B = u b(phi) (through every equilibrium the step
 * evaluates: cells, faces and ghosts, oracle_equilibrium_du).  The forward quantities are
 * recomputed exactly as in oracle_step; every stage is then transposed in
 * reverse order: cell update, face flux and Eq. 2.22, reconstruction
 * (Eqs. 2.19, 2.20, 2.26), ghost cells, Eqs. 2.21 / 2.13, phi = sum f.
 */
int oracle_adjoint_step(const oracle_problem *p, const double *f_in, const double *mu, double *lam,
                        double *dj_dalpha, double *dj_du) {
    if (!valid(p) || p->nsrc > 0) return -2; /* the adjoint covers the step without sources */
    workspace ws, *w = &ws;
    if (ws_alloc(w, p) != 0) { ws_free(w); return -1; }
    const int nx = p->nx, ny = p->ny, ex = nx + 2, ey = ny + 2;
    const size_t n = (size_t)nx * ny, ne = (size_t)ex * ey;
    const double h = 0.5 * p->dt, dt = p->dt, lam_t = relax_time(p);
    const double den1 = 2.0 * lam_t + dt, den2 = 2.0 * lam_t + h;
    const double a_bp = (2.0 * lam_t - h) / den1, b_bp = 3.0 * h / den1;
    const double a_tp = (2.0 * lam_t - dt) / den1, b_tp = 2.0 * dt / den1;
    const double a_f = 2.0 * lam_t / den2, b_f = h / den2;
    /* derivatives of the weights with respect to lambda */
    const double da_bp = 2.0 * (dt + h) / (den1 * den1), db_bp = -6.0 * h / (den1 * den1);
    const double da_tp = 4.0 * dt / (den1 * den1), db_tp = -4.0 * dt / (den1 * den1);
    const double da_f = 2.0 * h / (den2 * den2), db_f = -2.0 * h / (den2 * den2);
    const int xper = p->bc[WALL_W] == BC_PERIODIC, yper = p->bc[WALL_S] == BC_PERIODIC;
    double djdl = 0.0, djdu[2] = {0.0, 0.0};
    double dux[Q], duy[Q];

    /* forward recomputation: phi, feq, fbar^+ with halo */
    for (int k = 0; k < ny; k++)
        for (int j = 0; j < nx; j++) {
            size_t c = (size_t)k * nx + j;
            double ft[Q], feq[Q], fbp[Q], ftp[Q], phi = 0.0;
            for (int i = 0; i < Q; i++) { ft[i] = f_in[i * n + c]; phi += ft[i]; }
            oracle_equilibrium(p, phi, feq);
            oracle_cell_transforms(p, ft, feq, fbp, ftp);
            w->phi[c] = phi;
            for (int i = 0; i < Q; i++) {
                w->feq[i * n + c] = feq[i];
                EXT(w, i, k + 1, j + 1) = fbp[i];
            }
        }
    fill_halo(p, w);

    double *Pb = calloc(Q * ne, sizeof(double));   /* adjoint of fbar^+ on the extended grid */
    if (!Pb) { ws_free(w); return -1; }
#define PB(i, k, j) Pb[((size_t)(i) * ey + (size_t)(k)) * ex + (size_t)(j)]

    /* x-faces: recompute fbar, phi_b; then the adjoint of the face */
    for (int k = 0; k < ny; k++)
        for (int jf = 0; jf <= nx; jf++) {
            const int jl = jf, jr = jf + 1, ke = k + 1;
            const double xb = p->xf[jf], dxc = w->xc[jr] - w->xc[jl];
            const double wgt = (xb - w->xc[jl]) / dxc;
            const int wallW = !xper && jf == 0, wallE = !xper && jf == nx;
            double fbar[Q], gtl[Q], gtr[Q];
            for (int i = 0; i < Q; i++) {
                double gn = (EXT(w, i, ke, jr) - EXT(w, i, ke, jl)) / dxc;
                double val = EXT(w, i, ke, jl) + (xb - w->xc[jl]) * gn;
                double gt;
                if (wallW) gt = grad_y(w, w->fbp, i, ke, jr);
                else if (wallE) gt = grad_y(w, w->fbp, i, ke, jl);
                else gt = (1.0 - wgt) * grad_y(w, w->fbp, i, ke, jl) + wgt * grad_y(w, w->fbp, i, ke, jr);
                fbar[i] = val - h * (CX[i] * p->c * gn + CY[i] * p->c * gt);
                gtl[i] = wallW ? 0.0 : (wallE ? 1.0 : 1.0 - wgt); /* weight of the left G */
                gtr[i] = wallE ? 0.0 : (wallW ? 1.0 : wgt);       /* weight of the right G */
            }
            double phib = 0.0, feqb[Q], dfeqb[Q];
            for (int i = 0; i < Q; i++) phib += fbar[i];
            oracle_equilibrium(p, phib, feqb);
            oracle_equilibrium_deriv(p, phib, dfeqb);
            /* adjoint of the face values f_i: the update is ftp - dt/|V| (c_ix f_E dy - c_ix f_W dy + ...) */
            double fbarf[Q], s = 0.0;
            for (int i = 0; i < Q; i++) {
                double g = 0.0;
                if (jf >= 1) g -= dt / (p->xf[jf] - p->xf[jf - 1]) * CX[i] * p->c * mu[i * n + (size_t)k * nx + (jf - 1)];
                if (jf <= nx - 1) g += dt / (p->xf[jf + 1] - p->xf[jf]) * CX[i] * p->c * mu[i * n + (size_t)k * nx + jf];
                fbarf[i] = g;  /* dJ/d f_i at this face */
                djdl += g * (da_f * fbar[i] + db_f * feqb[i]);
                s += g * b_f * dfeqb[i];
            }
            oracle_equilibrium_du(p, phib, dux, duy);
            for (int i = 0; i < Q; i++) {
                djdu[0] += fbarf[i] * b_f * dux[i];
                djdu[1] += fbarf[i] * b_f * duy[i];
            }
            for (int i = 0; i < Q; i++) {
                const double fbb = a_f * fbarf[i] + s;  /* dJ/d fbar_i (Eq. 2.22 and phi_b = sum fbar) */
                const double cl = 1.0 - (xb - w->xc[jl]) / dxc + h * CX[i] * p->c / dxc;
                const double cr = (xb - w->xc[jl]) / dxc - h * CX[i] * p->c / dxc;
                PB(i, ke, jl) += cl * fbb;
                PB(i, ke, jr) += cr * fbb;
                const double gb = -h * CY[i] * p->c * fbb;  /* dJ/d gt */
                if (gtl[i] != 0.0) {
                    const double q = gb * gtl[i] / (w->yc[ke + 1] - w->yc[ke - 1]);
                    PB(i, ke + 1, jl) += q;
                    PB(i, ke - 1, jl) -= q;
                }
                if (gtr[i] != 0.0) {
                    const double q = gb * gtr[i] / (w->yc[ke + 1] - w->yc[ke - 1]);
                    PB(i, ke + 1, jr) += q;
                    PB(i, ke - 1, jr) -= q;
                }
            }
        }
    /* y-faces */
    for (int kf = 0; kf <= ny; kf++)
        for (int j = 0; j < nx; j++) {
            const int kl = kf, kr = kf + 1, je = j + 1;
            const double yb = p->yf[kf], dyc = w->yc[kr] - w->yc[kl];
            const double wgt = (yb - w->yc[kl]) / dyc;
            const int wallS = !yper && kf == 0, wallN = !yper && kf == ny;
            double fbar[Q], gtl[Q], gtr[Q];
            for (int i = 0; i < Q; i++) {
                double gn = (EXT(w, i, kr, je) - EXT(w, i, kl, je)) / dyc;
                double val = EXT(w, i, kl, je) + (yb - w->yc[kl]) * gn;
                double gt;
                if (wallS) gt = grad_x(w, w->fbp, i, kr, je);
                else if (wallN) gt = grad_x(w, w->fbp, i, kl, je);
                else gt = (1.0 - wgt) * grad_x(w, w->fbp, i, kl, je) + wgt * grad_x(w, w->fbp, i, kr, je);
                fbar[i] = val - h * (CX[i] * p->c * gt + CY[i] * p->c * gn);
                gtl[i] = wallS ? 0.0 : (wallN ? 1.0 : 1.0 - wgt);
                gtr[i] = wallN ? 0.0 : (wallS ? 1.0 : wgt);
            }
            double phib = 0.0, feqb[Q], dfeqb[Q];
            for (int i = 0; i < Q; i++) phib += fbar[i];
            oracle_equilibrium(p, phib, feqb);
            oracle_equilibrium_deriv(p, phib, dfeqb);
            double fbarf[Q], s = 0.0;
            for (int i = 0; i < Q; i++) {
                double g = 0.0;
                if (kf >= 1) g -= dt / (p->yf[kf] - p->yf[kf - 1]) * CY[i] * p->c * mu[i * n + (size_t)(kf - 1) * nx + j];
                if (kf <= ny - 1) g += dt / (p->yf[kf + 1] - p->yf[kf]) * CY[i] * p->c * mu[i * n + (size_t)kf * nx + j];
                fbarf[i] = g;
                djdl += g * (da_f * fbar[i] + db_f * feqb[i]);
                s += g * b_f * dfeqb[i];
            }
            oracle_equilibrium_du(p, phib, dux, duy);
            for (int i = 0; i < Q; i++) {
                djdu[0] += fbarf[i] * b_f * dux[i];
                djdu[1] += fbarf[i] * b_f * duy[i];
            }
            for (int i = 0; i < Q; i++) {
                const double fbb = a_f * fbarf[i] + s;
                const double cl = 1.0 - (yb - w->yc[kl]) / dyc + h * CY[i] * p->c / dyc;
                const double cr = (yb - w->yc[kl]) / dyc - h * CY[i] * p->c / dyc;
                PB(i, kl, je) += cl * fbb;
                PB(i, kr, je) += cr * fbb;
                const double gb = -h * CX[i] * p->c * fbb;
                if (gtl[i] != 0.0) {
                    const double q = gb * gtl[i] / (w->xc[je + 1] - w->xc[je - 1]);
                    PB(i, kl, je + 1) += q;
                    PB(i, kl, je - 1) -= q;
                }
                if (gtr[i] != 0.0) {
                    const double q = gb * gtr[i] / (w->xc[je + 1] - w->xc[je - 1]);
                    PB(i, kr, je + 1) += q;
                    PB(i, kr, je - 1) -= q;
                }
            }
        }
    /* ghosts, in the reverse order of fill_halo */
    double *phib_extra = calloc(n, sizeof(double));  /* dJ/d phi of interior cells through NEE ghosts */
    if (!phib_extra) { free(Pb); ws_free(w); return -1; }
    if (yper)
        for (int i = 0; i < Q; i++)
            for (int j = 0; j <= nx + 1; j++) {
                PB(i, ny, j) += PB(i, 0, j);
                PB(i, 1, j) += PB(i, ny + 1, j);
                PB(i, 0, j) = PB(i, ny + 1, j) = 0.0;
            }
    if (xper)
        for (int i = 0; i < Q; i++)
            for (int k = 0; k <= ny + 1; k++) {
                PB(i, k, nx) += PB(i, k, 0);
                PB(i, k, 1) += PB(i, k, nx + 1);
                PB(i, k, 0) = PB(i, k, nx + 1) = 0.0;
            }
    /* NEE ghost (jg,kg) from interior (ji,ki): P_g = feq(2 bv - phi_1) + P_1 - feq(phi_1) */
#define FOLD(jg, kg, ji, ki, bv)                                                                 \
    do {                                                                                         \
        const size_t c1 = (size_t)((ki) - 1) * nx + (size_t)((ji) - 1);                          \
        const double phi1 = w->phi[c1], phig = 2.0 * (bv) - phi1;                                \
        double d1[Q], dg[Q], u1x[Q], u1y[Q], ugx[Q], ugy[Q], acc = 0.0;                          \
        oracle_equilibrium_deriv(p, phi1, d1);                                                   \
        oracle_equilibrium_deriv(p, phig, dg);                                                   \
        oracle_equilibrium_du(p, phi1, u1x, u1y);                                                \
        oracle_equilibrium_du(p, phig, ugx, ugy);                                                \
        for (int i = 0; i < Q; i++) {                                                            \
            const double g = PB(i, (kg), (jg));                                                  \
            PB(i, (ki), (ji)) += g;                                                              \
            acc -= g * (dg[i] + d1[i]);                                                          \
            djdu[0] += g * (ugx[i] - u1x[i]);                                                    \
            djdu[1] += g * (ugy[i] - u1y[i]);                                                    \
            PB(i, (kg), (jg)) = 0.0;                                                             \
        }                                                                                        \
        phib_extra[c1] += acc;                                                                   \
    } while (0)
    if (!xper)
        for (int k = 1; k <= ny; k++) {
            FOLD(0, k, 1, k, p->bc_value[WALL_W]);
            FOLD(nx + 1, k, nx, k, p->bc_value[WALL_E]);
        }
    if (!yper)
        for (int j = 1; j <= nx; j++) {
            FOLD(j, 0, j, 1, p->bc_value[WALL_S]);
            FOLD(j, ny + 1, j, ny, p->bc_value[WALL_N]);
        }
#undef FOLD
    /* cells: P = a_bp f + b_bp feq(phi) (Eq. 2.21), T = a_tp f + b_tp feq(phi) (Eq. 2.13), phi = sum f */
    for (int k = 0; k < ny; k++)
        for (int j = 0; j < nx; j++) {
            const size_t c = (size_t)k * nx + j;
            double dfe[Q], acc = phib_extra[c];
            oracle_equilibrium_deriv(p, w->phi[c], dfe);
            oracle_equilibrium_du(p, w->phi[c], dux, duy);
            for (int i = 0; i < Q; i++) {
                const double pb = PB(i, k + 1, j + 1), tb = mu[i * n + c];
                acc += (b_bp * pb + b_tp * tb) * dfe[i];
                djdu[0] += (b_bp * pb + b_tp * tb) * dux[i];
                djdu[1] += (b_bp * pb + b_tp * tb) * duy[i];
                djdl += pb * (da_bp * f_in[i * n + c] + db_bp * w->feq[i * n + c]) +
                        tb * (da_tp * f_in[i * n + c] + db_tp * w->feq[i * n + c]);
            }
            for (int i = 0; i < Q; i++) lam[i * n + c] = a_bp * PB(i, k + 1, j + 1) + a_tp * mu[i * n + c] + acc;
        }
#undef PB
    if (dj_dalpha) *dj_dalpha += djdl / (p->c * p->c / 3.0);
    if (dj_du) {
        dj_du[0] += djdu[0];
        dj_du[1] += djdu[1];
    }
    free(phib_extra);
    free(Pb);
    ws_free(w);
    return 0;
}

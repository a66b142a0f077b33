/*
 * dugks3d_oracle.c -- plain, slow, FP64 CPU implementation of the DUGKS time
 * step for the three-dimensional NCDE with the D3Q15 (Eq. 2.28) or D3Q19
 * (Eq. 2.6) velocity set, written from the paper's Section 2.
 *
 * TEST INFRASTRUCTURE ONLY.  Like dugks_oracle.c (the 2-D oracle) this file
 * is the parity oracle of the 3-D path: only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it, and it shares no
 * code, header, table or helper with the CUDA library.
 *
 * The step follows the summary at the end of Section 2 in order, with
 * explicit intermediate arrays:
 *   1. phi = sum_i ft_i                                   (text after Eq. 2.13)
 *   2. feq_i(phi)                                         (Eq. 2.3)
 *   3. fbp = fbar^+ (Eq. 2.21) and ftp = ftilde^+ (Eq. 2.13)
 *   4. ghost / halo cells (periodic wrap, or the mirrored Dirichlet ghost)
 *   5. faces normal to x, y and z: value and slopes (Eqs. 2.19, 2.20), fbar at
 *      the face (Eq. 2.26), phi_b = sum_i fbar_i, feq(phi_b), f at the face
 *      (Eq. 2.22), flux (Eq. 2.9)
 *   6. cell update ft^{n+1} = ftp - dt/|V| J (Eq. 2.12 without sources)
 *
 * Readings (the 2-D oracle's, extended to 3-D): Eq. 2.15 read with its f_i
 * restored; lambda = alpha / c_s^2; C = u u int_0^phi b'(s)^2 ds or C = 0;
 * D = d(phi) I.  At a face the value and normal slope come from the two cells
 * (Eq. 2.20), and each of the two tangential slopes is (1-w) G_L + w G_R with
 * G the cell central difference; at a Dirichlet wall only the interior cell's
 * G is used.  Dirichlet ghost: x_g = 2 x_w - x_1, phi_g = 2 phi_w - phi_1,
 * fbp_g = feq(phi_g) + (fbp_1 - feq(phi_1)).  Walls ordered W, E (x), S, N
 * (y), B, T (z).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (with dugks_oracle.c)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 19

/* D3Q15 (Eq. 2.28) and D3Q19 (Eq. 2.6): directions in units of c, and weights. */
static const int C15[15][3] = {{0, 0, 0},   {1, 0, 0},    {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                               {0, 0, 1},   {0, 0, -1},   {1, 1, 1},   {1, 1, -1},  {1, -1, 1},
                               {-1, 1, 1},  {-1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}, {1, -1, -1}};
static const double W15[15] = {2.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9, 1.0 / 72,
                               1.0 / 72, 1.0 / 72, 1.0 / 72, 1.0 / 72, 1.0 / 72, 1.0 / 72, 1.0 / 72};
static const int C19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                               {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},  {-1, 0, -1}, {-1, 0, 1},
                               {1, 0, -1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
static const double W19[19] = {1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                               1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                               1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

typedef struct {
    int nx, ny, nz;
    const double *xf, *yf, *zf; /* face coordinates, increasing: nx+1, ny+1, nz+1 */
    int bc[6];                  /* W, E, S, N, B, T: 0 periodic, 1 Dirichlet */
    double bc_value[6];
    int lattice;                /* 15 or 19 */
    double c;
    double u[3];                /* B(phi) = u b(phi) */
    int nb;
    double b[8];
    double alpha;
    int nd;
    double d[8];                /* D = d(phi) I */
    int c_zero;
    double dt;
} oracle3_problem;

static int nq(const oracle3_problem *p) { return p->lattice == 15 ? 15 : 19; }
static int cv(const oracle3_problem *p, int i, int a) { return p->lattice == 15 ? C15[i][a] : C19[i][a]; }
static double wt(const oracle3_problem *p, int i) { return p->lattice == 15 ? W15[i] : W19[i]; }

static double poly3(int n, const double *a, double x) {
    double s = 0.0, pw = 1.0;
    for (int k = 0; k < n; k++) {
        s += a[k] * pw;
        pw *= x;
    }
    return s;
}

/* int_0^phi b'(s)^2 ds, term by term */
static double aux3(const oracle3_problem *p, double phi) {
    double s = 0.0;
    for (int k = 1; k < p->nb; k++)
        for (int l = 1; l < p->nb; l++) {
            int e = k + l - 1;
            s += (double)k * (double)l * p->b[k] * p->b[l] * pow(phi, (double)e) / (double)e;
        }
    return s;
}

/* Eq. 2.3: feq_i = w_i [phi + c_i.B/cs^2 + (cs^2 D + C - cs^2 phi I):(c_i c_i - cs^2 I)/(2 cs^4)] */
void oracle3_equilibrium(const oracle3_problem *p, double phi, double *feq) {
    const double cs2 = p->c * p->c / 3.0;
    const double bv = poly3(p->nb, p->b, phi), dv = poly3(p->nd, p->d, phi);
    const double cv_ = p->c_zero ? 0.0 : aux3(p, phi);
    double T[3][3];
    for (int a = 0; a < 3; a++)
        for (int e = 0; e < 3; e++) {
            const double delta = a == e ? 1.0 : 0.0;
            T[a][e] = cs2 * dv * delta + p->u[a] * p->u[e] * cv_ - cs2 * phi * delta;
        }
    for (int i = 0; i < nq(p); i++) {
        double ci[3];
        for (int a = 0; a < 3; a++) ci[a] = cv(p, i, a) * p->c;
        double cB = 0.0;
        for (int a = 0; a < 3; a++) cB += ci[a] * p->u[a] * bv;
        double contr = 0.0;
        for (int a = 0; a < 3; a++)
            for (int e = 0; e < 3; e++) contr += T[a][e] * (ci[a] * ci[e] - cs2 * (a == e ? 1.0 : 0.0));
        feq[i] = wt(p, i) * (phi + cB / cs2 + contr / (2.0 * cs2 * cs2));
    }
}

/* Section 4 opening: ft = feq(phi0); layout f[i][z][y][x]. */
void oracle3_init(const oracle3_problem *p, const double *phi0, double *f) {
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    for (size_t c = 0; c < n; c++) {
        double feq[QMAX];
        oracle3_equilibrium(p, phi0[c], feq);
        for (int i = 0; i < nq(p); i++) f[i * n + c] = feq[i];
    }
}

void oracle3_phi(const oracle3_problem *p, const double *f, double *phi) {
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    for (size_t c = 0; c < n; c++) {
        double s = 0.0;
        for (int i = 0; i < nq(p); i++) s += f[i * n + c];
        phi[c] = s;
    }
}

double oracle3_mass(const oracle3_problem *p, const double *f) {
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    double m = 0.0;
    for (int l = 0; l < p->nz; l++)
        for (int k = 0; k < p->ny; k++)
            for (int j = 0; j < p->nx; j++) {
                size_t c = ((size_t)l * p->ny + k) * p->nx + j;
                double s = 0.0;
                for (int i = 0; i < nq(p); i++) s += f[i * n + c];
                m += (p->xf[j + 1] - p->xf[j]) * (p->yf[k + 1] - p->yf[k]) * (p->zf[l + 1] - p->zf[l]) * s;
            }
    return m;
}

/* ------------------------------------------------------------------ */

typedef struct {
    int n[3], e[3];    /* interior and extended (1-cell halo) sizes per axis */
    double *xc[3];     /* extended centre coordinates per axis, index +1 */
    double *phi, *feq; /* interior */
    double *fbp;       /* [Q][ez][ey][ex] with halo */
    double *ftp;       /* interior [Q][nz][ny][nx] */
    double *flux[3];   /* face fluxes c_i.n f_i per axis: [Q][faces of that axis] */
} ws3;

static const double *face_coords(const oracle3_problem *p, int a) { return a == 0 ? p->xf : a == 1 ? p->yf : p->zf; }

static int ws3_alloc(ws3 *w, const oracle3_problem *p) {
    memset(w, 0, sizeof(*w));
    w->n[0] = p->nx; w->n[1] = p->ny; w->n[2] = p->nz;
    for (int a = 0; a < 3; a++) w->e[a] = w->n[a] + 2;
    const int Q = nq(p);
    const size_t n = (size_t)p->nx * p->ny * p->nz, ne = (size_t)w->e[0] * w->e[1] * w->e[2];
    for (int a = 0; a < 3; a++) {
        w->xc[a] = malloc(sizeof(double) * w->e[a]);
        if (!w->xc[a]) return -1;
        const double *f = face_coords(p, a);
        const int na = w->n[a];
        for (int j = 0; j < na; j++) w->xc[a][j + 1] = 0.5 * (f[j] + f[j + 1]);
        if (p->bc[2 * a] == 0) {
            const double L = f[na] - f[0];
            w->xc[a][0] = w->xc[a][na] - L;
            w->xc[a][na + 1] = w->xc[a][1] + L;
        } else {
            w->xc[a][0] = 2.0 * f[0] - w->xc[a][1];
            w->xc[a][na + 1] = 2.0 * f[na] - w->xc[a][na];
        }
        size_t nf = (size_t)(w->n[0] + (a == 0)) * (w->n[1] + (a == 1)) * (w->n[2] + (a == 2));
        w->flux[a] = malloc(sizeof(double) * Q * nf);
        if (!w->flux[a]) return -1;
    }
    w->phi = malloc(sizeof(double) * n);
    w->feq = malloc(sizeof(double) * Q * n);
    w->fbp = malloc(sizeof(double) * Q * ne);
    w->ftp = malloc(sizeof(double) * Q * n);
    return (w->phi && w->feq && w->fbp && w->ftp) ? 0 : -1;
}

static void ws3_free(ws3 *w) {
    for (int a = 0; a < 3; a++) { free(w->xc[a]); free(w->flux[a]); }
    free(w->phi); free(w->feq); free(w->fbp); free(w->ftp);
}

/* extended index (halo included) of cell (j, k, l), each in [-1, n] */
#define EIDX(w, j, k, l) ((((size_t)(l) + 1) * (w)->e[1] + ((size_t)(k) + 1)) * (w)->e[0] + ((size_t)(j) + 1))
#define EXT3(w, i, j, k, l) ((w)->fbp[(size_t)(i) * (w)->e[0] * (w)->e[1] * (w)->e[2] + EIDX(w, j, k, l)])

/* NEE ghost at extended (jg, kg, lg) mirroring interior (ji, ki, li) across a wall of value phiw */
static void nee3(const oracle3_problem *p, ws3 *w, int jg, int kg, int lg, int ji, int ki, int li, double phiw) {
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    const size_t c = ((size_t)li * p->ny + ki) * p->nx + ji;
    const double phig = 2.0 * phiw - w->phi[c];
    double feqg[QMAX];
    oracle3_equilibrium(p, phig, feqg);
    for (int i = 0; i < nq(p); i++) EXT3(w, i, jg, kg, lg) = feqg[i] + (EXT3(w, i, ji, ki, li) - w->feq[i * n + c]);
}

static void fill_halo3(const oracle3_problem *p, ws3 *w) {
    const int nx = p->nx, ny = p->ny, nz = p->nz, Q = nq(p);
    const int per[3] = {p->bc[0] == 0, p->bc[2] == 0, p->bc[4] == 0};
    /* poison the whole halo first: a halo cell that is read but neither set
     * nor wrapped below shows as NaN */
    for (int i = 0; i < Q; i++)
        for (int l = -1; l <= nz; l++)
            for (int k = -1; k <= ny; k++)
                for (int j = -1; j <= nx; j++)
                    if (j < 0 || j >= nx || k < 0 || k >= ny || l < 0 || l >= nz) EXT3(w, i, j, k, l) = NAN;
    /* Dirichlet ghosts on the interior ranges of the other two axes */
    if (!per[0])
        for (int l = 0; l < nz; l++)
            for (int k = 0; k < ny; k++) {
                nee3(p, w, -1, k, l, 0, k, l, p->bc_value[0]);
                nee3(p, w, nx, k, l, nx - 1, k, l, p->bc_value[1]);
            }
    if (!per[1])
        for (int l = 0; l < nz; l++)
            for (int j = 0; j < nx; j++) {
                nee3(p, w, j, -1, l, j, 0, l, p->bc_value[2]);
                nee3(p, w, j, ny, l, j, ny - 1, l, p->bc_value[3]);
            }
    if (!per[2])
        for (int k = 0; k < ny; k++)
            for (int j = 0; j < nx; j++) {
                nee3(p, w, j, k, -1, j, k, 0, p->bc_value[4]);
                nee3(p, w, j, k, nz, j, k, nz - 1, p->bc_value[5]);
            }
    /* periodic wraps over the full extended ranges, one axis after another */
    for (int i = 0; i < Q; i++) {
        if (per[0])
            for (int l = -1; l <= nz; l++)
                for (int k = -1; k <= ny; k++) {
                    EXT3(w, i, -1, k, l) = EXT3(w, i, nx - 1, k, l);
                    EXT3(w, i, nx, k, l) = EXT3(w, i, 0, k, l);
                }
        if (per[1])
            for (int l = -1; l <= nz; l++)
                for (int j = -1; j <= nx; j++) {
                    EXT3(w, i, j, -1, l) = EXT3(w, i, j, ny - 1, l);
                    EXT3(w, i, j, ny, l) = EXT3(w, i, j, 0, l);
                }
        if (per[2])
            for (int k = -1; k <= ny; k++)
                for (int j = -1; j <= nx; j++) {
                    EXT3(w, i, j, k, -1) = EXT3(w, i, j, k, nz - 1);
                    EXT3(w, i, j, k, nz) = EXT3(w, i, j, k, 0);
                }
    }
}

/* central difference of fbp along axis t at extended cell (j, k, l), velocity i:
 * (P(+1) - P(-1)) / (x(+1) - x(-1)) with x the extended centre coordinates */
static double grad3(const ws3 *w, int i, int t, int j, int k, int l) {
    const int dj = t == 0, dk = t == 1, dl = t == 2;
    const int it = t == 0 ? j : t == 1 ? k : l;
    return (EXT3(w, i, j + dj, k + dk, l + dl) - EXT3(w, i, j - dj, k - dk, l - dl)) /
           (w->xc[t][it + 2] - w->xc[t][it]);
}

static void step3(const oracle3_problem *p, ws3 *w, const double *f_in, double *f_out, int nthreads) {
    const int nx = p->nx, ny = p->ny, nz = p->nz, Q = nq(p);
    const size_t n = (size_t)nx * ny * nz;
    const double dt = p->dt, h = 0.5 * dt, lam = p->alpha / (p->c * p->c / 3.0);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    /* 1-3 */
#pragma omp parallel for schedule(static)
    for (int l = 0; l < nz; l++)
        for (int k = 0; k < ny; k++)
            for (int j = 0; j < nx; j++) {
                const size_t c = ((size_t)l * ny + k) * nx + j;
                double ft[QMAX], feq[QMAX], phi = 0.0;
                for (int i = 0; i < Q; i++) { ft[i] = f_in[i * n + c]; phi += ft[i]; }
                oracle3_equilibrium(p, phi, feq);
                w->phi[c] = phi;
                for (int i = 0; i < Q; i++) {
                    w->feq[i * n + c] = feq[i];
                    /* Eq. 2.21 and Eq. 2.13 */
                    EXT3(w, i, j, k, l) = (2.0 * lam - h) / (2.0 * lam + dt) * ft[i] + 3.0 * h / (2.0 * lam + dt) * feq[i];
                    w->ftp[i * n + c] = (2.0 * lam - dt) / (2.0 * lam + dt) * ft[i] + 2.0 * dt / (2.0 * lam + dt) * feq[i];
                }
            }
    /* 4 */
    fill_halo3(p, w);
    /* 5: faces normal to axis a; face index fidx in 0..n_a between cells fidx-1 and fidx */
    for (int a = 0; a < 3; a++) {
        const int per = p->bc[2 * a] == 0;
        const int na = w->n[a];
        const int fx = nx + (a == 0), fy = ny + (a == 1), fz = nz + (a == 2);
        const double *fc = face_coords(p, a);
        const int t1 = (a + 1) % 3, t2 = (a + 2) % 3; /* tangential axes */
#pragma omp parallel for schedule(static)
        for (int l = 0; l < fz; l++)
            for (int k = 0; k < fy; k++)
                for (int j = 0; j < fx; j++) {
                    const int fidx = a == 0 ? j : a == 1 ? k : l;
                    /* left cell (one back along a) and right cell (j, k, l) */
                    const int jl = j - (a == 0), kl = k - (a == 1), ll = l - (a == 2);
                    const double xl = w->xc[a][fidx], xr = w->xc[a][fidx + 1], xb = fc[fidx];
                    const double dxc = xr - xl, wgt = (xb - xl) / dxc;
                    double fbar[QMAX], f[QMAX], feqb[QMAX];
                    for (int i = 0; i < Q; i++) {
                        const double PL = EXT3(w, i, jl, kl, ll), PR = EXT3(w, i, j, k, l);
                        const double gn = (PR - PL) / dxc;      /* Eq. 2.20 slope */
                        const double val = PL + (xb - xl) * gn; /* Eq. 2.20 value */
                        double cdotg = cv(p, i, a) * p->c * gn;
                        for (int s = 0; s < 2; s++) {
                            const int t = s == 0 ? t1 : t2;
                            double g;
                            if (!per && fidx == 0)
                                g = grad3(w, i, t, j, k, l);    /* low wall: interior right cell */
                            else if (!per && fidx == na)
                                g = grad3(w, i, t, jl, kl, ll); /* high wall: interior left cell */
                            else
                                g = (1.0 - wgt) * grad3(w, i, t, jl, kl, ll) + wgt * grad3(w, i, t, j, k, l);
                            cdotg += cv(p, i, t) * p->c * g;
                        }
                        /* Eq. 2.19 + Eq. 2.26 */
                        fbar[i] = val - h * cdotg;
                    }
                    /* interface phi (text after Eq. 2.20), feq(phi_b), Eq. 2.22 */
                    double phib = 0.0;
                    for (int i = 0; i < Q; i++) phib += fbar[i];
                    oracle3_equilibrium(p, phib, feqb);
                    for (int i = 0; i < Q; i++) f[i] = 2.0 * lam / (2.0 * lam + h) * fbar[i] + h / (2.0 * lam + h) * feqb[i];
                    const size_t nf = (size_t)fx * fy * fz, fi = ((size_t)l * fy + k) * fx + j;
                    for (int i = 0; i < Q; i++) w->flux[a][(size_t)i * nf + fi] = cv(p, i, a) * p->c * f[i];
                }
    }
    /* 6: Eq. 2.12, J = sum over the six faces of (c_i . n) f_i |S| */
#pragma omp parallel for schedule(static)
    for (int l = 0; l < nz; l++)
        for (int k = 0; k < ny; k++)
            for (int j = 0; j < nx; j++) {
                const size_t c = ((size_t)l * ny + k) * nx + j;
                const double dx = p->xf[j + 1] - p->xf[j], dy = p->yf[k + 1] - p->yf[k], dz = p->zf[l + 1] - p->zf[l];
                const double area[3] = {dy * dz, dx * dz, dx * dy};
                for (int i = 0; i < Q; i++) {
                    double J = 0.0;
                    for (int a = 0; a < 3; a++) {
                        const int fx = nx + (a == 0), fy = ny + (a == 1), fz = nz + (a == 2);
                        const size_t nf = (size_t)fx * fy * fz;
                        const size_t lo = ((size_t)l * fy + k) * fx + j;
                        const size_t hi = ((size_t)(l + (a == 2)) * fy + (k + (a == 1))) * fx + (j + (a == 0));
                        J += (w->flux[a][(size_t)i * nf + hi] - w->flux[a][(size_t)i * nf + lo]) * area[a];
                    }
                    f_out[i * n + c] = w->ftp[i * n + c] - dt / (dx * dy * dz) * J;
                }
            }
}

static int valid3(const oracle3_problem *p) {
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || p->nb < 0 || p->nb > 8 || p->nd < 0 || p->nd > 8) return 0;
    if (p->lattice != 15 && p->lattice != 19) return 0;
    for (int a = 0; a < 3; a++)
        if ((p->bc[2 * a] == 0) != (p->bc[2 * a + 1] == 0)) return 0;
    return p->alpha > 0.0 && p->c > 0.0 && p->dt > 0.0;
}

int oracle3_step(const oracle3_problem *p, const double *f_in, double *f_out, int nthreads) {
    ws3 w;
    if (!valid3(p)) return -2;
    if (ws3_alloc(&w, p) != 0) { ws3_free(&w); return -1; }
    step3(p, &w, f_in, f_out, nthreads);
    ws3_free(&w);
    return 0;
}

int oracle3_run(const oracle3_problem *p, double *f, long nsteps, int nthreads) {
    const size_t sz = sizeof(double) * nq(p) * (size_t)p->nx * p->ny * p->nz;
    ws3 w;
    if (!valid3(p)) return -2;
    double *tmp = malloc(sz);
    if (!tmp || ws3_alloc(&w, p) != 0) { free(tmp); ws3_free(&w); return -1; }
    for (long s = 0; s < nsteps; s++) {
        step3(p, &w, f, tmp, nthreads);
        memcpy(f, tmp, sz);
    }
    ws3_free(&w);
    free(tmp);
    return 0;
}

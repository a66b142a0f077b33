// dugks_adjoint.cuh -- discrete adjoint of one DUGKS step (reverse mode of
// the step of Section 2 of arXiv:1906.11036), for gradients of a misfit of
// phi^N with respect to phi^0, the diffusion coefficient alpha and the
// velocity u of B = u b(phi).
//
// Given the forward state f = ftilde^n and mu = dJ/d ftilde^{n+1}, the
// kernels return lam = dJ/d ftilde^n and the explicit alpha- and
// u-derivatives of the step contracted with mu (alpha enters through
// lambda = alpha / c_s^2 in the weights of Eqs. 2.13, 2.21 and 2.22; u through
// every equilibrium the step evaluates, Eq. 2.3 with C = u u int b'^2:
// d feq_i / d u_a = A_ia b(phi) + B_ia Cint(phi), A_ia = 3 w_i e_ia / c,
// B_ia = w_i (9 e_ia (e_i.u) - 3 u_a) / c^2, e_i the unit direction).
//
//   adj_tile_kernel, per tile of cells: (P) recomputes the forward P = fbar^+
//     of its cells and halo (Eq. 2.21, mirrored ghosts); (faces) the forward face
//     value fbar (Eqs. 2.19, 2.20, 2.26), phi_b and feq(phi_b), takes the
//     adjoint g of the face flux from the two cells that use it (Eq. 2.12) and
//     forms the adjoint of fbar through Eq. 2.22:
//     A_i = a_f g_i + b_f sum_m g_m feq_m'(phi_b); (cells) gathers the adjoint
//     of P from the faces whose reconstruction used it (normal weights and the
//     transposed central differences of the tangential slopes) and transposes
//     Eqs. 2.21 and 2.13 and phi = sum f.
//   adj_wall_kernel : per cell next to a Dirichlet wall, folds the adjoint of
//     the mirrored NEE ghost beyond the wall back into the cell (linear in the
//     ghost's adjoint, so it is added to lam afterwards).
// Periodic faces 0 and nx (or ny) are the same physical face; both carry the
// adjoint of both neighbours, and each cell gathers it once.
#pragma once
#include "dugks_kernels.cuh"

namespace dugks {

template <typename T, int NC>
struct AdjConsts {
    T dfeq[Q][NC];  // d feq_i / d phi (i > 0); the rest velocity follows the zeroth moment
    T a_bp, b_bp, a_tp, b_tp, a_f, b_f;
    T da_bp, db_bp, da_tp, db_tp, da_f, db_f;  // derivatives of the weights with respect to lambda
    T bpoly[NC], cpoly[NC];                   // b(phi) and Cint(phi) = int_0^phi b'^2 (0 with C = 0)
    T Au[2][Q], Bu[2][Q];                     // d feq_i / d u_a = Au[a][i] b(phi) + Bu[a][i] Cint(phi)
};

template <typename T>
struct AdjArgs {
    const T* f;        // forward state ftilde^n, [Q][ny][nx] contiguous
    const T* mu;       // dJ/d ftilde^{n+1}
    T* lam;            // out: dJ/d ftilde^n
    T* Ax;             // x-face adjoints [Q][ny][nx+1]
    T* Ay;             // y-face adjoints [Q][ny+1][nx]
    double* partial;   // per-block partial sums: dJ/dlambda at [slot], dJ/du_x at [pstride + slot],
                       // dJ/du_y at [2 pstride + slot] (faces, cells, wall cells)
    long long pstride;
    int accumulate;    // 1: add to the partials (a reverse sweep sums them once at its end); 0: overwrite
    int want_u;        // 0: the u-derivative is not requested (its partials receive zeros)
};

// Neighbour index along one direction, for i in [-1, n]: the interior cell
// (periodic image) or, past a Dirichlet wall, the adjacent interior cell whose
// mirrored NEE ghost sits there.
struct Nb {
    int i;
    bool ghost;
};
__device__ __forceinline__ Nb nb_index(int i, int n, bool per) {
    if (i < 0) return per ? Nb{i + n, false} : Nb{0, true};
    if (i >= n) return per ? Nb{i - n, false} : Nb{n - 1, true};
    return Nb{i, false};
}

template <typename T, int NC>
__device__ __forceinline__ void dfeq_all(const AdjConsts<T, NC>& ka, T phi, T (&out)[Q]) {
    T s = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        T v = ka.dfeq[i][NC - 1];
#pragma unroll
        for (int m = NC - 2; m >= 0; --m) v = fma(v, phi, ka.dfeq[i][m]);
        out[i] = v;
        s += v;
    }
    out[0] = T(1) - s;
}

// d feq_i / d phi of one moving velocity (i > 0), as dfeq_all computes it
template <typename T, int NC>
__device__ __forceinline__ T dfeq_i(const AdjConsts<T, NC>& ka, int i, T phi) {
    T v = ka.dfeq[i][NC - 1];
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) v = fma(v, phi, ka.dfeq[i][m]);
    return v;
}

// polynomial sum_m c[m] x^m by Horner's rule
template <typename T, int NC>
__device__ __forceinline__ T poly_nc(const T (&c)[NC], T x) {
    T s = c[NC - 1];
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma(s, x, c[m]);
    return s;
}

// sum_i w_i d feq_i / d u_a at phi for a = x, y, over the velocities in `mask`
// (bit i: velocity i), added to du[0], du[1] in double
template <typename T, int NC>
__device__ __forceinline__ void add_du(const AdjConsts<T, NC>& ka, T phi, const T (&w)[Q], unsigned mask,
                                       double (&du)[2]) {
    const T bv = poly_nc<T, NC>(ka.bpoly, phi), cv = poly_nc<T, NC>(ka.cpoly, phi);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        T sa = T(0), sb = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (mask & (1u << i)) {
                sa = fma(w[i], ka.Au[a][i], sa);
                sb = fma(w[i], ka.Bu[a][i], sb);
            }
        du[a] += double(fma(bv, sa, cv * sb));
    }
}
__host__ __device__ constexpr unsigned xmask() { return (1u << 1) | (1u << 3) | (1u << 5) | (1u << 6) | (1u << 7) | (1u << 8); }
__host__ __device__ constexpr unsigned ymask() { return (1u << 2) | (1u << 4) | (1u << 5) | (1u << 6) | (1u << 7) | (1u << 8); }
constexpr unsigned kAllQ = (1u << Q) - 1u;

// The block's sums of v[0..2] (dJ/dlambda, dJ/du_x, dJ/du_y) into out[0], out[stride],
// out[2 stride] (one slot per block: no race), added to the slots or overwriting them.
__device__ __forceinline__ void block_partial3(const double (&v)[3], double* out, long long stride, int accumulate) {
    __shared__ double ws[3][32];
    double x[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x[q] += __shfl_xor_sync(0xffffffffu, x[q], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < 3; ++q) ws[q][threadIdx.x >> 5] = x[q];
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += ws[threadIdx.x][w];
        double* o = out + threadIdx.x * stride;
        *o = accumulate ? *o + s : s;
    }
}

// Cells next to a Dirichlet wall.  The mirrored NEE ghost beyond the wall has
// P_g = feq(2 bv - phi) + P - feq(phi) of this cell; its adjoint (the x- or
// y-face weights of the ghost, as in the cell gather of adj_tile_kernel) folds back into the cell.
// Everything the fold adds is linear in the ghost adjoints, so it is added to
// the lam that adj_tile_kernel wrote.  Threads enumerate rows 0 and ny-1 (when
// y has walls), then columns 0 and nx-1 of the remaining rows (when x has walls).
template <typename T, int NC>
__global__ void __launch_bounds__(128) adj_wall_kernel(const StepArgs<T, NC> a, const Consts<T, NC> k,
                                                       const AdjConsts<T, NC> ka, const AdjArgs<T> g,
                                                       const int first_partial) {
    const int nx = a.nx, ny = a.ny;
    const long long cplane = (long long)nx * ny;
    const long long xplane = (long long)(nx + 1) * ny, yplane = (long long)nx * (ny + 1);
    const int nrc = a.yper ? 0 : (ny > 1 ? 2 : 1) * nx;
    const int r0 = a.yper ? 0 : 1, r1 = a.yper ? ny : ny - 1;
    const int nr = max(0, r1 - r0);
    const int ncc = a.xper ? 0 : (nx > 1 ? 2 : 1) * nr;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double djdl = 0.0, du[2] = {0.0, 0.0};
    if (t < nrc + ncc) {
        int j, kr;
        if (t < nrc) {
            kr = t / nx == 0 ? 0 : ny - 1;
            j = t % nx;
        } else {
            const int u = t - nrc;
            j = u / nr == 0 ? 0 : nx - 1;
            kr = r0 + u % nr;
        }
        const long long c = (long long)kr * nx + j;
        const FaceM<T> fxW = a.fx[j + 1], fxE = a.fx[j + 2], fyS = a.fy[kr + 1], fyN = a.fy[kr + 2];
        const T* Ax0 = g.Ax + (long long)kr * (nx + 1) + j;  // x-faces j (+0) and j+1 (+1) of row kr
        const T* Ay0 = g.Ay + (long long)kr * nx + j;        // y-faces kr (+0) and kr+1 (+nx) of column j
        T ft[Q], fe[Q], dfe[Q], PG[Q];
        T phi = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            ft[i] = g.f[i * cplane + c];
            phi += ft[i];
            PG[i] = T(0);
        }
        feq_all(k, phi, fe);
        dfeq_all(ka, phi, dfe);
        T dphibar = T(0);
        auto fold = [&](const T (&Pg)[Q], T bv) {
            T dg[Q];
            dfeq_all(ka, T(2) * bv - phi, dg);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                PG[i] += Pg[i];
                dphibar -= Pg[i] * (dg[i] + dfe[i]);
            }
            if (g.want_u) add_du(ka, T(2) * bv - phi, Pg, kAllQ, du);  // feq(phi_g) of the ghost
        };
        if (!a.xper && j == 0) {  // west ghost: left cell of x-face 0; its P enters G^x(0, kr)
            T Pg[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = ((T(1) - fxW.w) + T(EX(i)) * fxW.hcd) * Ax0[i * xplane];
                if (EX(i) != 0)
                    v -= (-T(EX(i)) * k.hc) * a.cx[1].ig * (fyN.tl * Ay0[i * yplane + nx] + fyS.tr * Ay0[i * yplane]);
                Pg[i] = v;
            }
            fold(Pg, k.bcv[0]);
        }
        if (!a.xper && j == nx - 1) {  // east ghost: right cell of x-face nx; its P enters G^x(nx-1, kr)
            T Pg[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = (fxE.w - T(EX(i)) * fxE.hcd) * Ax0[i * xplane + 1];
                if (EX(i) != 0)
                    v += (-T(EX(i)) * k.hc) * a.cx[nx].ig * (fyN.tl * Ay0[i * yplane + nx] + fyS.tr * Ay0[i * yplane]);
                Pg[i] = v;
            }
            fold(Pg, k.bcv[1]);
        }
        if (!a.yper && kr == 0) {  // south ghost
            T Pg[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = ((T(1) - fyS.w) + T(EY(i)) * fyS.hcd) * Ay0[i * yplane];
                if (EY(i) != 0)
                    v -= (-T(EY(i)) * k.hc) * a.cy[1].ig * (fxE.tl * Ax0[i * xplane + 1] + fxW.tr * Ax0[i * xplane]);
                Pg[i] = v;
            }
            fold(Pg, k.bcv[2]);
        }
        if (!a.yper && kr == ny - 1) {  // north ghost
            T Pg[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = (fyN.w - T(EY(i)) * fyN.hcd) * Ay0[i * yplane + nx];
                if (EY(i) != 0)
                    v += (-T(EY(i)) * k.hc) * a.cy[ny].ig * (fxE.tl * Ax0[i * xplane + 1] + fxW.tr * Ax0[i * xplane]);
                Pg[i] = v;
            }
            fold(Pg, k.bcv[3]);
        }
        // the ghosts' share of Eq. 2.21's transpose (P enters through a_bp f + b_bp feq(phi))
        T s = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            dphibar += ka.b_bp * PG[i] * dfe[i];
            s += PG[i] * fma(ka.da_bp, ft[i], ka.db_bp * fe[i]);
        }
        djdl = double(s);
        if (g.want_u) {  // - feq(phi) of every ghost and b_bp feq(phi) of Eq. 2.21 through P of the cell
            T w[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) w[i] = (ka.b_bp - T(1)) * PG[i];
            add_du(ka, phi, w, kAllQ, du);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) g.lam[i * cplane + c] += fma(ka.a_bp, PG[i], dphibar);
    }
    const double v[3] = {djdl, du[0], du[1]};
    block_partial3(v, g.partial + first_partial + blockIdx.x, g.pstride, g.accumulate);
}

// The face and cell parts of the adjoint step in one launch.  A CTA of TX x TY
// threads owns the cells j0..j0+TX-1, k0..k0+TY-1.  It stages P (with the ghost
// transform) for a two-cell halo and mu for a one-cell halo in shared memory,
// computes the adjoints A of every face its cells gather from (x-faces j0..j0+TX
// of rows k0-1..k0+TY, y-faces k0..k0+TY of columns j0-1..j0+TX), then gathers
// the adjoint of P for each of its cells from those shared face adjoints.  A face's dJ/dlambda term is counted by the CTA that owns it (its cell
// range, plus the last face of the domain); with walls, owned faces are also
// written to Ax / Ay for adj_wall_kernel.
struct TileIdx {
    int i;      // interior index (wrapped), or the interior cell a ghost mirrors
    int state;  // 0 interior, 1 ghost (one cell beyond a Dirichlet wall), 2 beyond any use
};
__device__ __forceinline__ TileIdx tile_idx(int i, int n, bool per) {
    if (per) {
        i %= n;
        return TileIdx{i < 0 ? i + n : i, 0};
    }
    if (i >= 0 && i < n) return TileIdx{i, 0};
    if (i == -1) return TileIdx{0, 1};
    if (i == n) return TileIdx{n - 1, 1};
    return TileIdx{0, 2};
}

template <typename T, int TX, int TY>
struct AdjTile {
    static constexpr int PW = TX + 4, PH = TY + 4;  // P: columns j0-2.., rows k0-2..
    static constexpr int MW = TX + 2, MH = TY + 2;  // mu: columns j0-1.., rows k0-1..
    static constexpr int XW = TX + 1, XH = TY + 2;  // x-faces j0..j0+TX, rows k0-1..k0+TY
    static constexpr int YW = TX + 2, YH = TY + 1;  // y-faces k0..k0+TY, columns j0-1..j0+TX
    static constexpr size_t bytes() { return size_t(Q) * (PW * PH + MW * MH + XW * XH + YW * YH) * sizeof(T); }
};

template <typename T, int NC, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) adj_tile_kernel(const StepArgs<T, NC> a, const Consts<T, NC> k,
                                                           const AdjConsts<T, NC> ka, const AdjArgs<T> g,
                                                           const int write_faces) {
    using L = AdjTile<T, TX, TY>;
    extern __shared__ __align__(16) unsigned char adj_smem[];
    T* sP = reinterpret_cast<T*>(adj_smem);
    T* sMu = sP + Q * L::PW * L::PH;
    T* sAx = sMu + Q * L::MW * L::MH;
    T* sAy = sAx + Q * L::XW * L::XH;
    const int nx = a.nx, ny = a.ny;
    const long long cplane = (long long)nx * ny;
    const long long xplane = (long long)(nx + 1) * ny, yplane = (long long)nx * (ny + 1);
    const int j0 = blockIdx.x * TX, k0 = blockIdx.y * TY;
    const int tid = threadIdx.x, nthr = TX * TY;
    double djdl = 0.0, du[2] = {0.0, 0.0};

    // 1. P tile (two-cell halo) and mu tile (one-cell halo)
    for (int e = tid; e < L::PW * L::PH; e += nthr) {
        const int pc = e % L::PW, pr = e / L::PW;
        const TileIdx X = tile_idx(j0 - 2 + pc, nx, a.xper), Y = tile_idx(k0 - 2 + pr, ny, a.yper);
        T P[Q];
        if (X.state == 2 || Y.state == 2 || (X.state == 1 && Y.state == 1)) {
#pragma unroll
            for (int i = 0; i < Q; ++i) P[i] = T(0);  // beyond use, or a corner ghost (zero weights only)
        } else {  // P = fbar^+ (Eq. 2.21) from ftilde, and the mirrored ghost P_g = feq(2 bv - phi) + P - feq(phi)
            const long long c = (long long)Y.i * nx + X.i;
            T ft[Q], fe[Q];
            T phi = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                ft[i] = g.f[i * cplane + c];
                phi += ft[i];
            }
            feq_all(k, phi, fe);
#pragma unroll
            for (int i = 0; i < Q; ++i) P[i] = fma(k.a_bp, ft[i], k.b_bp * fe[i]);
            if (X.state == 1 || Y.state == 1) {
                const bool gx = X.state == 1;
                const T bv = gx ? (j0 - 2 + pc < 0 ? k.bcv[0] : k.bcv[1]) : (k0 - 2 + pr < 0 ? k.bcv[2] : k.bcv[3]);
                T fg[Q];
                feq_all(k, T(2) * bv - phi, fg);
#pragma unroll
                for (int i = 0; i < Q; ++i) P[i] = fg[i] + (P[i] - fe[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) sP[(i * L::PH + pr) * L::PW + pc] = P[i];
    }
    for (int e = tid; e < L::MW * L::MH; e += nthr) {
        const int mc = e % L::MW, mr = e / L::MW;
        const TileIdx X = tile_idx(j0 - 1 + mc, nx, a.xper), Y = tile_idx(k0 - 1 + mr, ny, a.yper);
        const bool real = X.state == 0 && Y.state == 0;
        const long long c = (long long)Y.i * nx + X.i;
#pragma unroll
        for (int i = 0; i < Q; ++i) sMu[(i * L::MH + mr) * L::MW + mc] = real ? g.mu[i * cplane + c] : T(0);
    }
    __syncthreads();

    auto Pt = [&](int i, int r, int c) -> T { return sP[(i * L::PH + r) * L::PW + c]; };
    auto Mt = [&](int i, int r, int c) -> T { return sMu[(i * L::MH + r) * L::MW + c]; };

    // 2a. x-face adjoints: face jf = j0 + xc between cells jf-1 and jf of row k0 - 1 + xr
    for (int e = tid; e < L::XW * L::XH; e += nthr) {
        const int xc = e % L::XW, xr = e / L::XW;
        const int jf = j0 + xc, row = k0 - 1 + xr;
        const TileIdx Rw = tile_idx(row, ny, a.yper);
        T A[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) A[i] = T(0);
        if (jf <= nx && Rw.state == 0) {
            const bool lghost = !a.xper && jf == 0, rghost = !a.xper && jf == nx;
            const FaceM<T> m = a.fx[jf + 1];
            const T ig = a.cy[Rw.i + 1].ig;
            const int pl = xc + 1, pr = xc + 2, prow = xr + 1;  // P tile coordinates of L, R
            T fb[Q];
            T phib = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T en = T(EX(i)), et = T(EY(i));
                const T GL = lghost ? T(0) : (Pt(i, prow + 1, pl) - Pt(i, prow - 1, pl)) * ig;
                const T GR = rghost ? T(0) : (Pt(i, prow + 1, pr) - Pt(i, prow - 1, pr)) * ig;
                fb[i] = ((T(1) - m.w) + en * m.hcd) * Pt(i, prow, pl) - et * k.hc * m.tl * GL +
                        (m.w - en * m.hcd) * Pt(i, prow, pr) - et * k.hc * m.tr * GR;
                phib += fb[i];
            }
            // feq and its derivative at phi_b: only the velocities crossing the face carry a flux adjoint
            T fe[Q], dfe[Q];
#pragma unroll
            for (int i = 1; i < Q; ++i)
                if (EX(i) != 0) {
                    fe[i] = feq_i(k, i, phib);
                    dfe[i] = dfeq_i(ka, i, phib);
                }
            const TileIdx Lc = tile_idx(jf - 1, nx, a.xper), Rc = tile_idx(jf, nx, a.xper);
            const T rL = lghost ? T(0) : a.cx[Lc.i + 1].r, rR = rghost ? T(0) : a.cx[Rc.i + 1].r;
            T gv[Q];
            T sg = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = T(0);
                if (EX(i) != 0) v = T(EX(i)) * (rR * Mt(i, xr, xc + 1) - rL * Mt(i, xr, xc));
                gv[i] = v;
                if (EX(i) != 0) sg += v * dfe[i];
            }
            T sdl = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                A[i] = fma(ka.a_f, gv[i], ka.b_f * sg);
                if (EX(i) != 0) sdl += gv[i] * fma(ka.da_f, fb[i], ka.db_f * fe[i]);
            }
            const bool owned = (xr >= 1 && xr <= TY && row < ny) && (xc < TX || jf == nx);
            if (owned && !(a.xper && jf == nx)) {  // a periodic face is counted once
                djdl += double(sdl);
                if (g.want_u) {  // Eq. 2.22: b_f feq(phi_b) of the crossing velocities
                    T w[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) w[i] = ka.b_f * gv[i];
                    add_du(ka, phib, w, xmask(), du);
                }
            }
            if (owned && write_faces) {
                T* Ag = g.Ax + (long long)row * (nx + 1) + jf;
#pragma unroll
                for (int i = 0; i < Q; ++i) Ag[i * xplane] = A[i];
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) sAx[(i * L::XH + xr) * L::XW + xc] = A[i];
    }
    // 2b. y-face adjoints: face kf = k0 + yr between rows kf-1 and kf of column j0 - 1 + yc
    for (int e = tid; e < L::YW * L::YH; e += nthr) {
        const int yc = e % L::YW, yr = e / L::YW;
        const int kf = k0 + yr, col = j0 - 1 + yc;
        const TileIdx Cw = tile_idx(col, nx, a.xper);
        T A[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) A[i] = T(0);
        if (kf <= ny && Cw.state == 0) {
            const bool lghost = !a.yper && kf == 0, rghost = !a.yper && kf == ny;
            const FaceM<T> m = a.fy[kf + 1];
            const T ig = a.cx[Cw.i + 1].ig;
            const int pc = yc + 1, pl = yr + 1, pr = yr + 2;  // P tile column, rows of L (below) and R
            T fb[Q];
            T phib = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T en = T(EY(i)), et = T(EX(i));
                const T GL = lghost ? T(0) : (Pt(i, pl, pc + 1) - Pt(i, pl, pc - 1)) * ig;
                const T GR = rghost ? T(0) : (Pt(i, pr, pc + 1) - Pt(i, pr, pc - 1)) * ig;
                fb[i] = ((T(1) - m.w) + en * m.hcd) * Pt(i, pl, pc) - et * k.hc * m.tl * GL +
                        (m.w - en * m.hcd) * Pt(i, pr, pc) - et * k.hc * m.tr * GR;
                phib += fb[i];
            }
            // feq and its derivative at phi_b: only the velocities crossing the face carry a flux adjoint
            T fe[Q], dfe[Q];
#pragma unroll
            for (int i = 1; i < Q; ++i)
                if (EY(i) != 0) {
                    fe[i] = feq_i(k, i, phib);
                    dfe[i] = dfeq_i(ka, i, phib);
                }
            const TileIdx Lr = tile_idx(kf - 1, ny, a.yper), Rr = tile_idx(kf, ny, a.yper);
            const T rL = lghost ? T(0) : a.cy[Lr.i + 1].r, rR = rghost ? T(0) : a.cy[Rr.i + 1].r;
            T gv[Q];
            T sg = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = T(0);
                if (EY(i) != 0) v = T(EY(i)) * (rR * Mt(i, yr + 1, yc) - rL * Mt(i, yr, yc));
                gv[i] = v;
                if (EY(i) != 0) sg += v * dfe[i];
            }
            T sdl = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                A[i] = fma(ka.a_f, gv[i], ka.b_f * sg);
                if (EY(i) != 0) sdl += gv[i] * fma(ka.da_f, fb[i], ka.db_f * fe[i]);
            }
            const bool owned = (yc >= 1 && yc <= TX && col < nx) && (yr < TY || kf == ny);
            if (owned && !(a.yper && kf == ny)) {
                djdl += double(sdl);
                if (g.want_u) {
                    T w[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) w[i] = ka.b_f * gv[i];
                    add_du(ka, phib, w, ymask(), du);
                }
            }
            if (owned && write_faces) {
                T* Ag = g.Ay + (long long)kf * nx + col;
#pragma unroll
                for (int i = 0; i < Q; ++i) Ag[i * yplane] = A[i];
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) sAy[(i * L::YH + yr) * L::YW + yc] = A[i];
    }
    __syncthreads();

    // 3. cells: gather the adjoint of P from the shared face adjoints
    const int tx = tid % TX, ty = tid / TX;
    const int j = j0 + tx, kr = k0 + ty;
    if (j < nx && kr < ny) {
        const long long t = (long long)kr * nx + j;
        const Nb xm = nb_index(j - 1, nx, a.xper), xp = nb_index(j + 1, nx, a.xper);
        const Nb ym = nb_index(kr - 1, ny, a.yper), yp = nb_index(kr + 1, ny, a.yper);
        const T igxm = xm.ghost ? T(0) : a.cx[xm.i + 1].ig, igxp = xp.ghost ? T(0) : a.cx[xp.i + 1].ig;
        const T igym = ym.ghost ? T(0) : a.cy[ym.i + 1].ig, igyp = yp.ghost ? T(0) : a.cy[yp.i + 1].ig;
        const FaceM<T> fxW = a.fx[j + 1], fxE = a.fx[j + 2], fyS = a.fy[kr + 1], fyN = a.fy[kr + 2];
        // x-face (face j0+xc, row k0-1+xr) and y-face (column j0-1+yc, face k0+yr) adjoints
        auto Ax = [&](int i, int xc, int xr) -> T { return sAx[(i * L::XH + xr) * L::XW + xc]; };
        auto Ay = [&](int i, int yc, int yr) -> T { return sAy[(i * L::YH + yr) * L::YW + yc]; };
        T Pb[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T ex = T(EX(i)), ey = T(EY(i));
            T v = ((T(1) - fxE.w) + ex * fxE.hcd) * Ax(i, tx + 1, ty + 1) + (fxW.w - ex * fxW.hcd) * Ax(i, tx, ty + 1) +
                  ((T(1) - fyN.w) + ey * fyN.hcd) * Ay(i, tx + 1, ty + 1) + (fyS.w - ey * fyS.hcd) * Ay(i, tx + 1, ty);
            if (EY(i) != 0) {
                const T c = -ey * k.hc;
                if (!ym.ghost) v += c * igym * (fxE.tl * Ax(i, tx + 1, ty) + fxW.tr * Ax(i, tx, ty));
                if (!yp.ghost) v -= c * igyp * (fxE.tl * Ax(i, tx + 1, ty + 2) + fxW.tr * Ax(i, tx, ty + 2));
            }
            if (EX(i) != 0) {
                const T c = -ex * k.hc;
                if (!xm.ghost) v += c * igxm * (fyN.tl * Ay(i, tx, ty + 1) + fyS.tr * Ay(i, tx, ty));
                if (!xp.ghost) v -= c * igxp * (fyN.tl * Ay(i, tx + 2, ty + 1) + fyS.tr * Ay(i, tx + 2, ty));
            }
            Pb[i] = v;
        }
        T ft[Q], mu[Q], fe[Q], dfe[Q];
        T phi = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            ft[i] = g.f[i * cplane + t];
            mu[i] = Mt(i, ty + 1, tx + 1);
            phi += ft[i];
        }
        feq_all(k, phi, fe);
        dfeq_all(ka, phi, dfe);
        T phibar = T(0), s = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            phibar += (ka.b_bp * Pb[i] + ka.b_tp * mu[i]) * dfe[i];
            s += Pb[i] * fma(ka.da_bp, ft[i], ka.db_bp * fe[i]) + mu[i] * fma(ka.da_tp, ft[i], ka.db_tp * fe[i]);
        }
        djdl += double(s);
        if (g.want_u) {  // Eqs. 2.21 and 2.13: b_bp feq(phi) in P and b_tp feq(phi) in ftilde^+
            T w[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) w[i] = fma(ka.b_bp, Pb[i], ka.b_tp * mu[i]);
            add_du(ka, phi, w, kAllQ, du);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) g.lam[i * cplane + t] = fma(ka.a_bp, Pb[i], fma(ka.a_tp, mu[i], phibar));
    }
    const double v[3] = {djdl, du[0], du[1]};
    block_partial3(v, g.partial + blockIdx.y * gridDim.x + blockIdx.x, g.pstride, g.accumulate);
}

// *dj_dalpha += (sum of the lambda partials) / c_s^2 and, if dj_du is set, dj_du[a] += (sum
// of the u_a partials), each in a fixed order (one block of 1024 threads).
__global__ void __launch_bounds__(1024) adj_sum_kernel(const double* __restrict__ partial, int n, long long stride,
                                                       double inv_cs2, double* __restrict__ dj_dalpha,
                                                       double* __restrict__ dj_du) {
    __shared__ double ws[32];
    for (int q = dj_dalpha ? 0 : 1; q < (dj_du ? 3 : 1); ++q) {
        const double* p = partial + q * stride;
        double acc = 0.0;
#pragma unroll 8
        for (int i = threadIdx.x; i < n; i += blockDim.x) acc += p[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < int(blockDim.x >> 5); ++w) s += ws[w];
            if (q == 0) *dj_dalpha += s * inv_cs2;
            else dj_du[q - 1] += s;
        }
        __syncthreads();
    }
}

// lam_i = g (the same for every velocity: phi = sum_i f_i)
template <typename T>
__global__ void broadcast_phi_adjoint(const T* __restrict__ gphi, T* __restrict__ lam, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const T v = gphi[c];
#pragma unroll
        for (int i = 0; i < Q; ++i) lam[i * n + c] = v;
    }
}

// dJ/dphi0 = sum_i feq_i'(phi0) lam_i (f^0 = feq(phi0), opening of Section 4); with upart set
// (3 gridDim.x doubles), the block's sums of sum_i lam_i d feq_i / d u_a(phi0) (f^0 depends on
// u too) go to upart[gridDim.x + blockIdx.x] and upart[2 gridDim.x + blockIdx.x], and 0 to
// upart[blockIdx.x].
template <typename T, int NC>
__global__ void __launch_bounds__(256) init_adjoint_kernel(const T* __restrict__ phi0, const T* __restrict__ lam,
                                                           T* __restrict__ gphi0, long long n,
                                                           const AdjConsts<T, NC> ka, double* __restrict__ upart) {
    double du[2] = {0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        T d[Q], l[Q];
        dfeq_all(ka, phi0[c], d);
        T s = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            l[i] = lam[i * n + c];
            s = fma(d[i], l[i], s);
        }
        gphi0[c] = s;
        if (upart) add_du(ka, phi0[c], l, kAllQ, du);
    }
    if (upart) {
        const double v[3] = {0.0, du[0], du[1]};
        block_partial3(v, upart + blockIdx.x, gridDim.x, 0);
    }
}

}  // namespace dugks

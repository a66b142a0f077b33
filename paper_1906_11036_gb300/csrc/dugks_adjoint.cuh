// dugks_adjoint.cuh -- discrete adjoint of one DUGKS step (reverse mode of
// the step of Section 2 of arXiv:1906.11036), for gradients of a misfit of
// phi^N with respect to phi^0 and the diffusion coefficient alpha.
//
// Given the forward state f = ftilde^n and mu = dJ/d ftilde^{n+1}, the two
// kernels return lam = dJ/d ftilde^n and the explicit alpha-derivative of the
// step contracted with mu (alpha enters through lambda = alpha / c_s^2 in the
// weights of Eqs. 2.13, 2.21 and 2.22).
//
//   adj_face_kernel : per face, recomputes the forward face value fbar
//     (Eqs. 2.19, 2.20, 2.26), phi_b and feq(phi_b), takes the adjoint g of
//     the face flux from the two cells that use it (Eq. 2.12) and returns the
//     adjoint of fbar through Eq. 2.22: A_i = a_f g_i + b_f sum_m g_m feq_m'(phi_b).
//   adj_cell_kernel : per cell, gathers the adjoint of P = fbar^+ from the
//     faces whose reconstruction used it (normal weights and the transposed
//     central differences of the tangential slopes) and transposes Eqs. 2.21
//     and 2.13 and phi = sum f.
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
};

template <typename T>
struct AdjArgs {
    const T* f;        // forward state ftilde^n, [Q][ny][nx] contiguous
    const T* mu;       // dJ/d ftilde^{n+1}
    T* lam;            // out: dJ/d ftilde^n
    T* Ax;             // x-face adjoints [Q][ny][nx+1]
    T* Ay;             // y-face adjoints [Q][ny+1][nx]
    T* P;              // forward fbar^+ of every cell [Q][ny][nx] (adj_p_kernel)
    T* phi;            // forward phi of every cell [ny][nx]
    double* partial;   // per-block partial sums of dJ/dlambda (faces, cells, wall cells)
    int accumulate;    // 1: add to the partials (a reverse sweep sums them once at its end); 0: overwrite
};

// Forward P = fbar^+ (Eq. 2.21) and phi of every cell, once per adjoint step.
template <typename T, int NC>
__global__ void __launch_bounds__(256) adj_p_kernel(const StepArgs<T, NC> a, const Consts<T, NC> k, const AdjArgs<T> g) {
    const long long n = (long long)a.nx * a.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        T ft[Q], fe[Q];
        T phi = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            ft[i] = g.f[i * n + c];
            phi += ft[i];
        }
        feq_all(k, phi, fe);
#pragma unroll
        for (int i = 0; i < Q; ++i) g.P[i * n + c] = fma(k.a_bp, ft[i], k.b_bp * fe[i]);
        g.phi[c] = phi;
    }
}

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

// P of cell c from the P buffer, or of the mirrored NEE ghost next to it:
// P_g = feq(2 bv - phi) + P - feq(phi).
template <typename T, int NC>
__device__ __forceinline__ void load_P(const Consts<T, NC>& k, const AdjArgs<T>& g, long long n, long long c,
                                       bool ghost, T bv, T (&P)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) P[i] = g.P[i * n + c];
    if (ghost) {
        const T phi = g.phi[c];
        T fe[Q], fg[Q];
        feq_all(k, phi, fe);
        feq_all(k, T(2) * bv - phi, fg);
#pragma unroll
        for (int i = 0; i < Q; ++i) P[i] = fg[i] + (P[i] - fe[i]);
    }
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

template <typename T>
__device__ __forceinline__ void block_partial(double v, double* out, int accumulate) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += ws[w];
        *out = accumulate ? *out + s : s;  // each block owns its slot: no race
    }
}

// Grid (ceil((nx+1)/blockDim.x), rows, 2): blockIdx.z = 0 for x-faces (threads
// along jf, rows kc), 1 for y-faces (threads along jc, rows kf).
template <typename T, int NC>
__global__ void __launch_bounds__(128) adj_face_kernel(const StepArgs<T, NC> a, const Consts<T, NC> k,
                                                       const AdjConsts<T, NC> ka, const AdjArgs<T> g) {
    const int nx = a.nx, ny = a.ny;
    const bool xface = blockIdx.z == 0;
    const long long cplane = (long long)nx * ny;
    const long long aplane = xface ? (long long)(nx + 1) * ny : (long long)nx * (ny + 1);
    const int along = blockIdx.x * blockDim.x + threadIdx.x;
    const int nalong = xface ? nx + 1 : nx, nrows = xface ? ny : ny + 1;
    const int n = xface ? nx : ny, nt = xface ? ny : nx;  // extents along the face normal and tangent
    const bool per = xface ? a.xper : a.yper, tper = xface ? a.yper : a.xper;
    const T bvL = xface ? k.bcv[0] : k.bcv[2], bvR = xface ? k.bcv[1] : k.bcv[3];
    const T bvm = xface ? k.bcv[2] : k.bcv[0], bvp = xface ? k.bcv[3] : k.bcv[1];
    double djdl = 0.0;
    if (along < nalong) {
        for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
            const int fidx = xface ? along : row;  // face index along its normal
            const int tc = xface ? row : along;    // tangential index of its two cells
            auto cell = [&](int inorm, int itan) -> long long {
                return xface ? (long long)itan * nx + inorm : (long long)inorm * nx + itan;
            };
            const Nb L = nb_index(fidx - 1, n, per), R = nb_index(fidx, n, per);
            const Nb Tm = nb_index(tc - 1, nt, tper), Tp = nb_index(tc + 1, nt, tper);
            const FaceM<T> m = xface ? a.fx[fidx + 1] : a.fy[fidx + 1];
            const T ig = xface ? a.cy[tc + 1].ig : a.cx[tc + 1].ig;
            // forward: P of the two cells and their tangential slopes (none for a ghost)
            T PL[Q], PR[Q], GL[Q], GR[Q], tA[Q], tB[Q];
            load_P(k, g, cplane, cell(L.i, tc), L.ghost, bvL, PL);
            load_P(k, g, cplane, cell(R.i, tc), R.ghost, bvR, PR);
#pragma unroll
            for (int i = 0; i < Q; ++i) { GL[i] = T(0); GR[i] = T(0); }
            if (!L.ghost) {
                load_P(k, g, cplane, cell(L.i, Tp.i), Tp.ghost, bvp, tA);
                load_P(k, g, cplane, cell(L.i, Tm.i), Tm.ghost, bvm, tB);
#pragma unroll
                for (int i = 0; i < Q; ++i) GL[i] = (tA[i] - tB[i]) * ig;
            }
            if (!R.ghost) {
                load_P(k, g, cplane, cell(R.i, Tp.i), Tp.ghost, bvp, tA);
                load_P(k, g, cplane, cell(R.i, Tm.i), Tm.ghost, bvm, tB);
#pragma unroll
                for (int i = 0; i < Q; ++i) GR[i] = (tA[i] - tB[i]) * ig;
            }
            T fb[Q];
            T phib = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T en = T(xface ? EX(i) : EY(i)), et = T(xface ? EY(i) : EX(i));
                fb[i] = ((T(1) - m.w) + en * m.hcd) * PL[i] - et * k.hc * m.tl * GL[i] + (m.w - en * m.hcd) * PR[i] -
                        et * k.hc * m.tr * GR[i];
                phib += fb[i];
            }
            T fe[Q], dfe[Q];
            feq_all(k, phib, fe);
            dfeq_all(ka, phib, dfe);
            // the two cells that use this face's flux (both neighbours for a periodic boundary face)
            const long long offL = cell(L.i, tc), offR = cell(R.i, tc);
            const T rL = L.ghost ? T(0) : (xface ? a.cx[L.i + 1].r : a.cy[L.i + 1].r);
            const T rR = R.ghost ? T(0) : (xface ? a.cx[R.i + 1].r : a.cy[R.i + 1].r);
            T gv[Q];
            T sg = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T en = T(xface ? EX(i) : EY(i));
                T v = T(0);
                if (en != T(0)) {
                    if (!R.ghost) v += rR * g.mu[i * cplane + offR];
                    if (!L.ghost) v -= rL * g.mu[i * cplane + offL];
                    v *= en;
                }
                gv[i] = v;
                sg += v * dfe[i];
            }
            T* A = xface ? g.Ax + (long long)row * (nx + 1) + along : g.Ay + (long long)row * nx + along;
            T s = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                A[i * aplane] = fma(ka.a_f, gv[i], ka.b_f * sg);
                s += gv[i] * fma(ka.da_f, fb[i], ka.db_f * fe[i]);
            }
            if (!(per && fidx == n)) djdl += double(s);  // a periodic face is counted once in dJ/dlambda
        }
    }
    block_partial<T>(djdl, g.partial + (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x, g.accumulate);
}

// Grid (ceil(nx/blockDim.x), rows): threads along j, blocks over rows kr.
template <typename T, int NC>
__global__ void __launch_bounds__(128, 4) adj_cell_kernel(const StepArgs<T, NC> a, const Consts<T, NC> k,
                                                       const AdjConsts<T, NC> ka, const AdjArgs<T> g,
                                                       const int face_blocks) {
    const int nx = a.nx, ny = a.ny;
    const long long cplane = (long long)nx * ny;
    const long long xplane = (long long)(nx + 1) * ny, yplane = (long long)nx * (ny + 1);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    double djdl = 0.0;
    if (j < nx) {
        const Nb xm = nb_index(j - 1, nx, a.xper), xp = nb_index(j + 1, nx, a.xper);
        const T igxm = xm.ghost ? T(0) : a.cx[xm.i + 1].ig, igxp = xp.ghost ? T(0) : a.cx[xp.i + 1].ig;
        const FaceM<T> fxW = a.fx[j + 1], fxE = a.fx[j + 2];
        for (int kr = blockIdx.y; kr < ny; kr += gridDim.y) {
            const long long t = (long long)kr * nx + j;
            const Nb ym = nb_index(kr - 1, ny, a.yper), yp = nb_index(kr + 1, ny, a.yper);
            const T igym = ym.ghost ? T(0) : a.cy[ym.i + 1].ig, igyp = yp.ghost ? T(0) : a.cy[yp.i + 1].ig;
            const FaceM<T> fyS = a.fy[kr + 1], fyN = a.fy[kr + 2];
            // x-face adjoints of faces j, j+1 in rows kr, kr-1, kr+1; y-face adjoints of
            // faces kr, kr+1 (offset nx) in columns j, j-1, j+1
            const T* Ax0 = g.Ax + (long long)kr * (nx + 1) + j;
            const T* Axm = g.Ax + (long long)ym.i * (nx + 1) + j;
            const T* Axp = g.Ax + (long long)yp.i * (nx + 1) + j;
            const T* Ay0 = g.Ay + (long long)kr * nx + j;
            const T* Aym = g.Ay + (long long)kr * nx + xm.i;
            const T* Ayp = g.Ay + (long long)kr * nx + xp.i;
            T Pb[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T ex = T(EX(i)), ey = T(EY(i));
                const T* ax = Ax0 + i * xplane;
                const T* ay = Ay0 + i * yplane;
                // normal weights of this cell in its four faces
                T v = ((T(1) - fxE.w) + ex * fxE.hcd) * ax[1] + (fxW.w - ex * fxW.hcd) * ax[0] +
                      ((T(1) - fyN.w) + ey * fyN.hcd) * ay[nx] + (fyS.w - ey * fyS.hcd) * ay[0];
                // tangential: this P enters G^y of the cells above and below, used by their x-faces
                if (EY(i) != 0) {
                    const T c = -ey * k.hc;
                    if (!ym.ghost) v += c * igym * (fxE.tl * Axm[i * xplane + 1] + fxW.tr * Axm[i * xplane]);
                    if (!yp.ghost) v -= c * igyp * (fxE.tl * Axp[i * xplane + 1] + fxW.tr * Axp[i * xplane]);
                }
                // and G^x of the cells left and right, used by their y-faces
                if (EX(i) != 0) {
                    const T c = -ex * k.hc;
                    if (!xm.ghost) v += c * igxm * (fyN.tl * Aym[i * yplane + nx] + fyS.tr * Aym[i * yplane]);
                    if (!xp.ghost) v -= c * igxp * (fyN.tl * Ayp[i * yplane + nx] + fyS.tr * Ayp[i * yplane]);
                }
                Pb[i] = v;
            }
            // forward cell quantities
            T ft[Q], mu[Q], fe[Q], dfe[Q];
            T phi = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                ft[i] = g.f[i * cplane + t];
                mu[i] = g.mu[i * cplane + t];
                phi += ft[i];
            }
            feq_all(k, phi, fe);
            dfeq_all(ka, phi, dfe);
            T phibar = T(0);
            // P = a_bp f + b_bp feq(phi) (Eq. 2.21), Fp = a_tp f + b_tp feq(phi) (Eq. 2.13), phi = sum f
            T s = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                phibar += (ka.b_bp * Pb[i] + ka.b_tp * mu[i]) * dfe[i];
                s += Pb[i] * fma(ka.da_bp, ft[i], ka.db_bp * fe[i]) + mu[i] * fma(ka.da_tp, ft[i], ka.db_tp * fe[i]);
            }
            djdl += double(s);
#pragma unroll
            for (int i = 0; i < Q; ++i) g.lam[i * cplane + t] = fma(ka.a_bp, Pb[i], fma(ka.a_tp, mu[i], phibar));
        }
    }
    block_partial<T>(djdl, g.partial + face_blocks + blockIdx.y * gridDim.x + blockIdx.x, g.accumulate);
}

// Cells next to a Dirichlet wall.  The mirrored NEE ghost beyond the wall has
// P_g = feq(2 bv - phi) + P - feq(phi) of this cell; its adjoint (the x- or
// y-face weights of the ghost, as in adj_cell_kernel) folds back into the cell.
// Everything the fold adds is linear in the ghost adjoints, so it is added to
// the lam that adj_cell_kernel wrote.  Threads enumerate rows 0 and ny-1 (when
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
    double djdl = 0.0;
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
#pragma unroll
        for (int i = 0; i < Q; ++i) g.lam[i * cplane + c] += fma(ka.a_bp, PG[i], dphibar);
    }
    block_partial<T>(djdl, g.partial + first_partial + blockIdx.x, g.accumulate);
}

// *dj_dalpha += (sum of the partials) / c_s^2, in a fixed order (one block of 1024).
__global__ void __launch_bounds__(1024) adj_sum_kernel(const double* __restrict__ partial, int n, double inv_cs2,
                                                       double* __restrict__ dj_dalpha) {
    double acc = 0.0;
#pragma unroll 8
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += ws[w];
        *dj_dalpha += s * inv_cs2;
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

// dJ/dphi0 = sum_i feq_i'(phi0) lam_i (f^0 = feq(phi0), opening of Section 4)
template <typename T, int NC>
__global__ void init_adjoint_kernel(const T* __restrict__ phi0, const T* __restrict__ lam, T* __restrict__ gphi0,
                                    long long n, const AdjConsts<T, NC> ka) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        T d[Q];
        dfeq_all(ka, phi0[c], d);
        T s = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) s = fma(d[i], lam[i * n + c], s);
        gphi0[c] = s;
    }
}

}  // namespace dugks

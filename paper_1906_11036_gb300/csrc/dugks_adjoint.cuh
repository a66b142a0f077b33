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
//     central differences of the tangential slopes), folds the mirrored NEE
//     ghosts back into their interior cells, and transposes Eqs. 2.21 and
//     2.13 and phi = sum f.
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
    double* partial;   // per-block partial sums of dJ/dlambda (faces, then cells)
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

// P at extended cell (jj, kk) from the P buffer: interior, periodic image, or the
// mirrored NEE ghost P_g = feq(2 bv - phi) + P - feq(phi) of the adjacent interior cell.
template <typename T, int NC>
__device__ void buf_P(const StepArgs<T, NC>& a, const Consts<T, NC>& k, const AdjArgs<T>& g, int jj, int kk,
                      T (&P)[Q]) {
    if (a.xper) jj = (jj + a.nx) % a.nx;
    if (a.yper) kk = (kk + a.ny) % a.ny;
    const bool gx = jj < 0 || jj >= a.nx, gy = kk < 0 || kk >= a.ny;
    if (gx && gy) {  // corner ghost: only ever multiplied by a zero weight
#pragma unroll
        for (int i = 0; i < Q; ++i) P[i] = T(0);
        return;
    }
    const int js = gx ? (jj < 0 ? 0 : a.nx - 1) : jj;
    const int ks = gy ? (kk < 0 ? 0 : a.ny - 1) : kk;
    const long long n = (long long)a.nx * a.ny, c = (long long)ks * a.nx + js;
#pragma unroll
    for (int i = 0; i < Q; ++i) P[i] = g.P[i * n + c];
    if (gx || gy) {
        const T phi = g.phi[c];
        const T bv = gx ? (jj < 0 ? k.bcv[0] : k.bcv[1]) : (kk < 0 ? k.bcv[2] : k.bcv[3]);
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
__device__ __forceinline__ void block_partial(double v, double* out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += ws[w];
        *out = s;
    }
}

// One thread per face: x-faces first ((nx+1) * ny of them), then y-faces (nx * (ny+1)).
template <typename T, int NC>
__global__ void __launch_bounds__(128) adj_face_kernel(const StepArgs<T, NC> a, const Consts<T, NC> k,
                                                       const AdjConsts<T, NC> ka, const AdjArgs<T> g) {
    const int nx = a.nx, ny = a.ny;
    const long long nxf = (long long)(nx + 1) * ny, nyf = (long long)nx * (ny + 1);
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double djdl = 0.0;
    const long long cplane = (long long)nx * ny;
    if (t < nxf + nyf) {
        const bool xface = t < nxf;
        int jf = 0, kf = 0, jc = 0, kc = 0;  // face index along its normal, and the row/column it lies in
        if (xface) { kc = int(t / (nx + 1)); jf = int(t % (nx + 1)); }
        else { const long long u = t - nxf; kf = int(u / nx); jc = int(u % nx); }
        const int fidx = xface ? jf : kf;
        const int n = xface ? nx : ny;
        const bool per = xface ? a.xper : a.yper;
        const FaceM<T> m = xface ? a.fx[jf + 1] : a.fy[kf + 1];
        // forward: P of the two cells and their tangential slopes
        T PL[Q], PR[Q], GL[Q], GR[Q], tmpA[Q], tmpB[Q];
        if (xface) {
            buf_P(a, k, g, jf - 1, kc, PL);
            buf_P(a, k, g, jf, kc, PR);
        } else {
            buf_P(a, k, g, jc, kf - 1, PL);
            buf_P(a, k, g, jc, kf, PR);
        }
        const bool lghost = !per && fidx == 0, rghost = !per && fidx == n;
#pragma unroll
        for (int i = 0; i < Q; ++i) { GL[i] = T(0); GR[i] = T(0); }
        if (!lghost) {
            if (xface) {
                buf_P(a, k, g, jf - 1, kc + 1, tmpA);
                buf_P(a, k, g, jf - 1, kc - 1, tmpB);
            } else {
                buf_P(a, k, g, jc + 1, kf - 1, tmpA);
                buf_P(a, k, g, jc - 1, kf - 1, tmpB);
            }
            const T ig = xface ? a.cy[kc + 1].ig : a.cx[jc + 1].ig;
#pragma unroll
            for (int i = 0; i < Q; ++i) GL[i] = (tmpA[i] - tmpB[i]) * ig;
        }
        if (!rghost) {
            if (xface) {
                buf_P(a, k, g, jf, kc + 1, tmpA);
                buf_P(a, k, g, jf, kc - 1, tmpB);
            } else {
                buf_P(a, k, g, jc + 1, kf, tmpA);
                buf_P(a, k, g, jc - 1, kf, tmpB);
            }
            const T ig = xface ? a.cy[kc + 1].ig : a.cx[jc + 1].ig;
#pragma unroll
            for (int i = 0; i < Q; ++i) GR[i] = (tmpA[i] - tmpB[i]) * ig;
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
        int cl = fidx - 1, cr = fidx;
        if (per) { cl = (cl + n) % n; cr = cr % n; }
        const bool hasL = cl >= 0 && cl < n, hasR = cr >= 0 && cr < n;
        const long long offL = xface ? (long long)kc * nx + cl : (long long)cl * nx + jc;
        const long long offR = xface ? (long long)kc * nx + cr : (long long)cr * nx + jc;
        const T rL = hasL ? (xface ? a.cx[cl + 1].r : a.cy[cl + 1].r) : T(0);
        const T rR = hasR ? (xface ? a.cx[cr + 1].r : a.cy[cr + 1].r) : T(0);
        T gv[Q];
        T sg = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T en = T(xface ? EX(i) : EY(i));
            T v = T(0);
            if (en != T(0)) {
                if (hasR) v += rR * g.mu[i * cplane + offR];
                if (hasL) v -= rL * g.mu[i * cplane + offL];
                v *= en;
            }
            gv[i] = v;
            sg += v * dfe[i];
        }
        const bool count = !(per && fidx == n);  // a periodic face is counted once in dJ/dlambda
        T* A = xface ? g.Ax + (long long)kc * (nx + 1) + jf : g.Ay + (long long)kf * nx + jc;
        const long long aplane = xface ? (long long)(nx + 1) * ny : (long long)nx * (ny + 1);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            A[i * aplane] = fma(ka.a_f, gv[i], ka.b_f * sg);
            if (count) djdl += double(gv[i]) * double(fma(ka.da_f, fb[i], ka.db_f * fe[i]));
        }
    }
    block_partial<T>(djdl, g.partial + blockIdx.x);
}

// One thread per cell.
template <typename T, int NC>
__global__ void __launch_bounds__(128) adj_cell_kernel(const StepArgs<T, NC> a, const Consts<T, NC> k,
                                                       const AdjConsts<T, NC> ka, const AdjArgs<T> g,
                                                       const int face_blocks) {
    const int nx = a.nx, ny = a.ny;
    const long long cplane = (long long)nx * ny;
    const long long xplane = (long long)(nx + 1) * ny, yplane = (long long)nx * (ny + 1);
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double djdl = 0.0;
    if (t < cplane) {
        const int kr = int(t / nx), j = int(t % nx);
        auto Ax = [&](int i, int jf, int kk) -> T {  // x-face adjoint, zero outside a Dirichlet row range
            if (kk < 0 || kk >= ny) {
                if (!a.yper) return T(0);
                kk = (kk + ny) % ny;
            }
            return g.Ax[i * xplane + (long long)kk * (nx + 1) + jf];
        };
        auto Ay = [&](int i, int jj, int kf) -> T {
            if (jj < 0 || jj >= nx) {
                if (!a.xper) return T(0);
                jj = (jj + nx) % nx;
            }
            return g.Ay[i * yplane + (long long)kf * nx + jj];
        };
        auto igy = [&](int kk) -> T { return a.cy[((kk + ny) % ny) + 1].ig; };
        auto igx = [&](int jj) -> T { return a.cx[((jj + nx) % nx) + 1].ig; };
        const FaceM<T> fxW = a.fx[j + 1], fxE = a.fx[j + 2], fyS = a.fy[kr + 1], fyN = a.fy[kr + 2];
        T Pb[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T ex = T(EX(i)), ey = T(EY(i));
            // normal weights of this cell in its four faces
            T v = ((T(1) - fxE.w) + ex * fxE.hcd) * Ax(i, j + 1, kr) + (fxW.w - ex * fxW.hcd) * Ax(i, j, kr) +
                  ((T(1) - fyN.w) + ey * fyN.hcd) * Ay(i, j, kr + 1) + (fyS.w - ey * fyS.hcd) * Ay(i, j, kr);
            // tangential: this P enters G^y of the cells above and below, used by their x-faces
            if (EY(i) != 0) {
                const T c = -ey * k.hc;
                if (a.yper || kr - 1 >= 0)
                    v += c * igy(kr - 1) * (fxE.tl * Ax(i, j + 1, kr - 1) + fxW.tr * Ax(i, j, kr - 1));
                if (a.yper || kr + 1 < ny)
                    v -= c * igy(kr + 1) * (fxE.tl * Ax(i, j + 1, kr + 1) + fxW.tr * Ax(i, j, kr + 1));
            }
            // and G^x of the cells left and right, used by their y-faces
            if (EX(i) != 0) {
                const T c = -ex * k.hc;
                if (a.xper || j - 1 >= 0)
                    v += c * igx(j - 1) * (fyN.tl * Ay(i, j - 1, kr + 1) + fyS.tr * Ay(i, j - 1, kr));
                if (a.xper || j + 1 < nx)
                    v -= c * igx(j + 1) * (fyN.tl * Ay(i, j + 1, kr + 1) + fyS.tr * Ay(i, j + 1, kr));
            }
            Pb[i] = v;
        }
        // forward cell quantities
        T ft[Q], fe[Q], dfe[Q];
        T phi = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            ft[i] = g.f[i * cplane + t];
            phi += ft[i];
        }
        feq_all(k, phi, fe);
        dfeq_all(ka, phi, dfe);
        T phibar = T(0);
        // mirrored NEE ghosts: P_g = feq(2 bv - phi) + P - feq(phi) (Dirichlet walls)
        auto fold = [&](const T (&Pg)[Q], T bv) {
            T dg[Q];
            dfeq_all(ka, T(2) * bv - phi, dg);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                Pb[i] += Pg[i];
                phibar -= Pg[i] * (dg[i] + dfe[i]);
            }
        };
        if (!a.xper && j == 0) {  // west ghost: left cell of x-face 0; its P enters G^x(0, kr)
            T Pg[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = ((T(1) - fxW.w) + T(EX(i)) * fxW.hcd) * Ax(i, 0, kr);
                if (EX(i) != 0)
                    v -= (-T(EX(i)) * k.hc) * igx(0) * (fyN.tl * Ay(i, 0, kr + 1) + fyS.tr * Ay(i, 0, kr));
                Pg[i] = v;
            }
            fold(Pg, k.bcv[0]);
        }
        if (!a.xper && j == nx - 1) {  // east ghost: right cell of x-face nx; its P enters G^x(nx-1, kr)
            T Pg[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = (fxE.w - T(EX(i)) * fxE.hcd) * Ax(i, nx, kr);
                if (EX(i) != 0)
                    v += (-T(EX(i)) * k.hc) * igx(nx - 1) * (fyN.tl * Ay(i, nx - 1, kr + 1) + fyS.tr * Ay(i, nx - 1, kr));
                Pg[i] = v;
            }
            fold(Pg, k.bcv[1]);
        }
        if (!a.yper && kr == 0) {  // south ghost
            T Pg[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = ((T(1) - fyS.w) + T(EY(i)) * fyS.hcd) * Ay(i, j, 0);
                if (EY(i) != 0)
                    v -= (-T(EY(i)) * k.hc) * igy(0) * (fxE.tl * Ax(i, j + 1, 0) + fxW.tr * Ax(i, j, 0));
                Pg[i] = v;
            }
            fold(Pg, k.bcv[2]);
        }
        if (!a.yper && kr == ny - 1) {  // north ghost
            T Pg[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = (fyN.w - T(EY(i)) * fyN.hcd) * Ay(i, j, ny);
                if (EY(i) != 0)
                    v += (-T(EY(i)) * k.hc) * igy(ny - 1) * (fxE.tl * Ax(i, j + 1, ny - 1) + fxW.tr * Ax(i, j, ny - 1));
                Pg[i] = v;
            }
            fold(Pg, k.bcv[3]);
        }
        // P = a_bp f + b_bp feq(phi) (Eq. 2.21), Fp = a_tp f + b_tp feq(phi) (Eq. 2.13), phi = sum f
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T mu = g.mu[i * cplane + t];
            phibar += (ka.b_bp * Pb[i] + ka.b_tp * mu) * dfe[i];
            djdl += double(Pb[i]) * double(fma(ka.da_bp, ft[i], ka.db_bp * fe[i])) +
                    double(mu) * double(fma(ka.da_tp, ft[i], ka.db_tp * fe[i]));
        }
#pragma unroll
        for (int i = 0; i < Q; ++i)
            g.lam[i * cplane + t] = fma(ka.a_bp, Pb[i], fma(ka.a_tp, g.mu[i * cplane + t], phibar));
    }
    block_partial<T>(djdl, g.partial + face_blocks + blockIdx.x);
}

// *dj_dalpha += (sum of the partials) / c_s^2, in a fixed order.
__global__ void __launch_bounds__(256) adj_sum_kernel(const double* __restrict__ partial, int n, double inv_cs2,
                                                      double* __restrict__ dj_dalpha) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[8];
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

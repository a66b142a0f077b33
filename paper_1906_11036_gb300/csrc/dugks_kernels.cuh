// dugks_kernels.cuh -- the DUGKS step kernels (arXiv:1906.11036, Section 2,
// step summary at the end of the section), plus initialisation and the
// phi / mass reduction.
//
//   naive_step  : one thread per cell; recomputes P = fbar^+ of its 3x3
//                 neighbourhood straight from global memory.  A simple
//                 cross-check of the fused kernel.
//   fused_step  : the production kernel.  One warp owns a strip of 30
//                 columns (plus one halo column on each side) and a segment
//                 of rows, and marches up the segment one row at a time.
//                 Each row of ftilde (all nine planes) arrives in shared
//                 memory by one 3-D TMA copy, several rows ahead, so ftilde
//                 is read once and written once per step.  P of the last
//                 rows, the y-face flux of the row below and the lower half
//                 of the next y-face stay in registers; x-neighbours exchange
//                 their halves of the x-face by warp shuffles.
#pragma once
#include <cuda.h>

#include "dugks_device.cuh"

namespace dugks {

template <typename T, int NC>
struct StepArgs {
    const T* fin;
    T* fout;
    int nx, ny;
    long long pitch;  // elements per row of one plane
    long long plane;  // elements per plane = pitch * ny
    int xper, yper;   // periodic flags per direction
    const FaceM<T>* fx;  // x-faces f = -1 .. nx+1 at index f+1
    const FaceM<T>* fy;  // y-faces f = -1 .. ny+1 at index f+1
    const CellM<T>* cx;  // columns j = -1 .. nx at index j+1
    const CellM<T>* cy;  // rows    k = -1 .. ny at index k+1
    int* err;            // device error word (bit 0: TMA wait timed out)
};

// Source F(x, t, phi) = sum_k exp(rate_k t) phi^power_k S_k(x) (Eq. 2.1) with
// R_i = w_i c_i.u b'(phi) F / c_s^2 (Eq. 2.3 as Remark 3 reduces it for
// C = int B'B' dphi).  The time derivatives in Eqs. 2.12 and 2.18 are the
// backward differences (S^n - S^{n-1}) / dt, so per cell
//   at the interface (Eq. 2.18): S + h/2 dS/dt = S^n + (S^n - S^{n-1}) / 4,
//   in the update    (Eq. 2.12): S + dt/2 dS/dt = (3 S^n - S^{n-1}) / 2.
// Both enter linearly: the interface term is added to P = fbar^+ before the
// face reconstruction (Eqs. 2.19, 2.20 are linear and identical for fbar^+,
// R and F), the update term to Fp = ftilde^+.  S^{n-1} comes from
// phi^{n-1}, kept in a history buffer.
template <typename T>
struct SrcArgs {
    int nterms;
    int first;            // 1: no history yet (S^{n-1} = S^n)
    int power[8];         // terms in ascending order of power
    int dpow[8];          // power[k] - power[k-1] (power[-1] = 0)
    T en[8], ep[8];       // exp(rate_k t_n), exp(rate_k t_{n-1})
    T db[8];              // b'(phi) coefficients, lowest order first
    int ndb;
    T kP_g[Q], kP_f[Q];   // per velocity: 2lh/(2l+h) w_i c_i.u / c_s^2 and h w_i
    T kU_g[Q], kU_f[Q];   // per velocity: dt w_i c_i.u / c_s^2 and dt w_i
    const T* field;       // S_k, [nterms][ny][nx] contiguous
    long long fplane;     // nx * ny
    const T* hin;         // phi^{n-1} [ny][nx]
    T* hout;              // phi^n [ny][nx]
    // velocity-pair path: fields and history in pitched planes staged by TMA with ftilde
    const T* aux_in;      // [nterms + 1][ny][pitch]: S_k, then phi^{n-1}
    T* aux_out;           // same layout; its last plane receives phi^n
    long long aux_plane;  // elements per plane (pitch * ny)
    int aux_box;          // bytes of one aux TMA box (nterms + 1 planes of one row)
    int stage_bytes;      // bytes of one ring stage: ftilde box + aux box (128-byte multiples)
};

// L1 prefetch of the source fields and the history of cell c (a few rows ahead of use)
template <typename T>
__device__ __forceinline__ void prefetch_source(const SrcArgs<T>& sa, long long c) {
    for (int q = 0; q < sa.nterms; ++q)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(sa.field + q * sa.fplane + c));
    if (!sa.first) asm volatile("prefetch.global.L1 [%0];" ::"l"(sa.hin + c));
}

// adds the source terms of cell c (index into the [ny][nx] arrays) with phi^n = phi;
// S^{n-1} from phi^{n-1} (on the first step the host passes ep = en and phi^{n-1} = phi^n)
template <typename T>
__device__ __forceinline__ void add_source(const SrcArgs<T>& sa, long long c, T phi, T (&P)[Q], T (&Fp)[Q],
                                           bool write_hist) {
    const T phio = sa.first ? phi : sa.hin[c];
    if (write_hist) sa.hout[c] = phi;
    // every field load is issued before any is used
    T Sv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) Sv[q] = q < sa.nterms ? sa.field[q * sa.fplane + c] : T(0);
    T Fn = T(0), Fo = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q >= sa.nterms) break;
        const T S = Sv[q];
        T xn = sa.en[q] * S, xo = sa.ep[q] * S;
        for (int m = 0; m < sa.power[q]; ++m) {
            xn *= phi;
            xo *= phio;
        }
        Fn += xn;
        Fo += xo;
    }
    T dn = T(0), dO = T(0);  // b'(phi^n), b'(phi^{n-1})
    for (int m = sa.ndb - 1; m >= 0; --m) {
        dn = fma(dn, phi, sa.db[m]);
        dO = fma(dO, phio, sa.db[m]);
    }
    const T gn = dn * Fn, go = dO * Fo;
    const T Ft = Fn + T(0.25) * (Fn - Fo), gt = gn + T(0.25) * (gn - go);
    const T Fa = T(1.5) * Fn - T(0.5) * Fo, ga = T(1.5) * gn - T(0.5) * go;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        P[i] += fma(sa.kP_g[i], gt, sa.kP_f[i] * Ft);
        Fp[i] += fma(sa.kU_g[i], ga, sa.kU_f[i] * Fa);
    }
}

// ---------------------------------------------------------------------------
// naive cross-check kernel
// ---------------------------------------------------------------------------

// P = fbar^+ at extended cell (jj, kk): interior, periodic image, or the
// mirrored ghost with non-equilibrium extrapolation at a Dirichlet wall.
template <typename T, int NC>
__device__ void naive_P(const StepArgs<T, NC>& a, const Consts<T, NC>& k, int jj, int kk, T (&P)[Q]) {
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
    T ft[Q], fe[Q];
    T phi = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        ft[i] = a.fin[i * a.plane + ks * a.pitch + js];
        phi += ft[i];
    }
    feq_all(k, phi, fe);
#pragma unroll
    for (int i = 0; i < Q; ++i) P[i] = fma(k.a_bp, ft[i], k.b_bp * fe[i]);
    if (gx || gy) {
        const T bv = gx ? (jj < 0 ? k.bcv[0] : k.bcv[1]) : (kk < 0 ? k.bcv[2] : k.bcv[3]);
        T fg[Q];
        feq_all(k, T(2) * bv - phi, fg);
#pragma unroll
        for (int i = 0; i < Q; ++i) P[i] = fg[i] + (P[i] - fe[i]);
    }
}

template <typename T, int NC>
__device__ void naive_cell(const StepArgs<T, NC>& a, const Consts<T, NC>& k, const int j, const int kr);

template <typename T, int NC>
__global__ void __launch_bounds__(128) naive_step(const StepArgs<T, NC> a, const Consts<T, NC> k) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.nx) return;
    for (int kr = blockIdx.y; kr < a.ny; kr += gridDim.y) naive_cell(a, k, j, kr);
}

template <typename T, int NC>
__device__ void naive_cell(const StepArgs<T, NC>& a, const Consts<T, NC>& k, const int j, const int kr) {
    T P[3][3][Q];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) naive_P(a, k, j + c - 1, kr + b - 1, P[b][c]);
    // tangential slopes: Gy at columns j-1, j, j+1 of row kr; Gx at rows kr-1, kr, kr+1 of column j
    T Gy[3][Q], Gx[3][Q];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int jj = j + c - 1;
        const bool ghost = !a.xper && (jj < 0 || jj >= a.nx);
        const T ig = a.cy[kr + 1].ig;
#pragma unroll
        for (int i = 0; i < Q; ++i) Gy[c][i] = ghost ? T(0) : (P[2][c][i] - P[0][c][i]) * ig;
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const int kk = kr + b - 1;
        const bool ghost = !a.yper && (kk < 0 || kk >= a.ny);
        const T ig = a.cx[j + 1].ig;
#pragma unroll
        for (int i = 0; i < Q; ++i) Gx[b][i] = ghost ? T(0) : (P[b][2][i] - P[b][0][i]) * ig;
    }
    T fW[6], fE[6], fS[6], fN[6], fb[Q];
    // x-faces: west (columns j-1 | j) and east (j | j+1)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const FaceM<T> m = a.fx[j + 1 + side];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T ex = T(EX(i)), ey = T(EY(i));
            fb[i] = ((T(1) - m.w) + ex * m.hcd) * P[1][side][i] - ey * k.hc * m.tl * Gy[side][i] +
                    (m.w - ex * m.hcd) * P[1][side + 1][i] - ey * k.hc * m.tr * Gy[side + 1][i];
        }
        if (side == 0) face_original<T, NC, true>(k, fb, fW);
        else face_original<T, NC, true>(k, fb, fE);
    }
    // y-faces: south (rows kr-1 | kr) and north (kr | kr+1)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const FaceM<T> m = a.fy[kr + 1 + side];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T ex = T(EX(i)), ey = T(EY(i));
            fb[i] = ((T(1) - m.w) + ey * m.hcd) * P[side][1][i] - ex * k.hc * m.tl * Gx[side][i] +
                    (m.w - ey * m.hcd) * P[side + 1][1][i] - ex * k.hc * m.tr * Gx[side + 1][i];
        }
        if (side == 0) face_original<T, NC, false>(k, fb, fS);
        else face_original<T, NC, false>(k, fb, fN);
    }
    // cell update (Eq. 2.12 without sources, Fp from Eq. 2.13)
    T ft[Q], fe[Q];
    T phi = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        ft[i] = a.fin[i * a.plane + kr * a.pitch + j];
        phi += ft[i];
    }
    feq_all(k, phi, fe);
    const T rx = a.cx[j + 1].r, ry = a.cy[kr + 1].r;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T v = fma(k.a_tp, ft[i], k.b_tp * fe[i]);
        if (XSLOT(i) >= 0) v -= T(EX(i)) * rx * (fE[XSLOT(i)] - fW[XSLOT(i)]);
        if (YSLOT(i) >= 0) v -= T(EY(i)) * ry * (fN[YSLOT(i)] - fS[YSLOT(i)]);
        a.fout[i * a.plane + kr * a.pitch + j] = v;
    }
}

// ---------------------------------------------------------------------------
// fused streaming kernel
// ---------------------------------------------------------------------------

// One warp owns WI = 30 interior columns of one row segment, plus one halo
// column on each side (lanes 0 and 31); lane l holds column xw - 1 + l.
// Warps are independent: each has its own ring of S shared-memory stages
// filled by 3-D TMA copies (one row of all nine planes per copy) and its own
// mbarriers, and exchanges neighbour values with warp shuffles only.
template <typename T>
struct WarpLayout {
    static constexpr int WI = 30;                       // interior columns per warp
    static constexpr int ALIGN = 16 / int(sizeof(T));   // TMA x-coordinate granule (16 bytes)
    static constexpr int BOXW = 32 + ALIGN;             // columns per TMA box row
    static constexpr int BOX_BYTES = Q * BOXW * int(sizeof(T));
    static constexpr int STAGE_BYTES = ((BOX_BYTES + 127) / 128) * 128;
    static size_t bytes(int stages) { return size_t(stages) * (STAGE_BYTES + 8) + 128; }
};

enum ColRole { ROLE_IN = 0, ROLE_GHOST_W, ROLE_GHOST_E, ROLE_WRAP_W, ROLE_WRAP_E, ROLE_OUT };

template <typename T>
__device__ __forceinline__ T shfl_dn(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_up(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }

// b_bp feq_i(x) and b_f feq_i(x) by Horner's rule (coefficients read straight from the
// constant bank; i must be a compile-time constant after unrolling)
template <typename T, int NC>
__device__ __forceinline__ T hbp_i(const Consts<T, NC>& k, int i, T x) {
    T s = k.hbp[i][NC - 1];
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma(s, x, k.hbp[i][m]);
    return s;
}
template <typename T, int NC>
__device__ __forceinline__ T hf_i(const Consts<T, NC>& k, int i, T x) {
    T s = k.hf[i][NC - 1];
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma(s, x, k.hf[i][m]);
    return s;
}

template <typename T, int NC, bool EDGE, bool SRC>
__device__ __forceinline__ void warp_rows(const CUtensorMap* tin, const StepArgs<T, NC>& a, const Consts<T, NC>& k,
                                          unsigned char* stages, uint64_t* bars, const int S, const int lane,
                                          const int xw, const int y0, const int y1, const SrcArgs<T>* sa) {
    using L = WarpLayout<T>;
    const int nx = a.nx, ny = a.ny;
    const int j = xw - 1 + lane;
    const int xs = (xw - 1) & ~(L::ALIGN - 1);
    const int R = y1 - y0 + 2;  // rows r = y0-1 .. y1 pass through the pipeline

    int role = ROLE_IN, scol = j;
    if (EDGE) {
        if (j >= 0 && j < nx) { role = ROLE_IN; scol = j; }
        else if (j == -1) { role = a.xper ? ROLE_WRAP_W : ROLE_GHOST_W; scol = a.xper ? nx - 1 : 0; }
        else if (j == nx) { role = a.xper ? ROLE_WRAP_E : ROLE_GHOST_E; scol = a.xper ? 0 : nx - 1; }
        else { role = ROLE_OUT; scol = 0; }
    }
    const bool from_smem = !EDGE || role == ROLE_IN || role == ROLE_GHOST_W || role == ROLE_GHOST_E;
    const bool ghost_col = EDGE && (role == ROLE_GHOST_W || role == ROLE_GHOST_E);
    const bool updates = (!EDGE || role == ROLE_IN) && lane >= 1 && lane <= L::WI;
    const int jm = EDGE ? min(max(j, -1), nx) : j;
    const FaceM<T> fW = a.fx[jm + 1], fE = a.fx[jm + 2];
    const CellM<T> cxj = a.cx[jm + 1];
    const T bvx = role == ROLE_GHOST_W ? k.bcv[0] : k.bcv[1];
    const int soff = scol - xs;

    // x-face weights of this cell, for e_x = -1, 0, +1: as the left cell of its east face and
    // as the right cell of its west face; tangential weights h c tl and h c tr
    T axL[3], axR[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        axL[e] = (T(1) - fE.w) + T(e - 1) * fE.hcd;
        axR[e] = fW.w - T(e - 1) * fW.hcd;
    }
    const T gxL = k.hc * fE.tl, gxR = k.hc * fW.tr;
    const T igx_in = cxj.ig, rx = cxj.r;

    auto src_row = [&](int r) -> int {
        if (r < 0) return a.yper ? r + ny : 0;
        if (r >= ny) return a.yper ? r - ny : ny - 1;
        return r;
    };
    if (lane == 0) {
        for (int q = 0; q < min(S, R); ++q) {
            mbar_arrive_expect_tx(&bars[q], uint32_t(L::BOX_BYTES));
            tma_load_3d(stages + size_t(q) * L::STAGE_BYTES, tin, &bars[q], xs, src_row(y0 - 1 + q), 0);
        }
    }
    int s = 0, issued = min(S, R), consumed = 0;
    uint32_t ph = 0;

    // next row of ftilde from the pipeline; refills the stage it frees
    auto load_row = [&](int r, T (&ft)[Q]) -> bool {
        const bool ok = mbar_wait_bounded(&bars[s], ph, 2000000000ull);
        if (__any_sync(0xffffffffu, !ok)) return false;
        if (from_smem) {
            const T* st = reinterpret_cast<const T*>(stages + size_t(s) * L::STAGE_BYTES) + soff;
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = st[i * L::BOXW];
        } else if (role != ROLE_OUT) {
            const long long base = (long long)src_row(r) * a.pitch + scol;
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = a.fin[i * a.plane + base];
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = T(0);
        }
        __syncwarp();
        if (issued < R) {
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[s], uint32_t(L::BOX_BYTES));
                tma_load_3d(stages + size_t(s) * L::STAGE_BYTES, tin, &bars[s], xs, src_row(r + S), 0);
            }
            ++issued;
        }
        if (++s == S) { s = 0; ph ^= 1u; }
        ++consumed;
        return true;
    };
    // P = fbar^+ (Eq. 2.21, with b_bp folded into the equilibrium polynomials) and
    // Fp = ftilde^+ = P + (P - ft)/3 (Eq. 2.23); ghost cells by the NEE reading
    auto cell_row = [&](int r, const T (&ft)[Q], T (&P)[Q], T (&Fp)[Q]) {
        T phi = ft[0];
#pragma unroll
        for (int i = 1; i < Q; ++i) phi += ft[i];
        T hs = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const T h = hbp_i(k, i, phi);
            P[i] = fma(k.a_bp, ft[i], h);
            hs += h;
        }
        P[0] = fma(k.a_bp, ft[0], fma(k.b_bp, phi, -hs));  // rest velocity via the zeroth moment
#pragma unroll
        for (int i = 0; i < Q; ++i) Fp[i] = fma(k.third, P[i] - ft[i], P[i]);
        const bool ghost_row = !a.yper && (r < 0 || r >= ny);
        if (SRC && !(EDGE && role == ROLE_OUT)) {  // a ghost takes the source of the interior cell it mirrors
            if (r + 4 <= y1) prefetch_source(*sa, (long long)src_row(r + 4) * nx + scol);
            add_source(*sa, (long long)src_row(r) * nx + scol, phi, P, Fp, updates && r >= y0 && r < y1);
        }
        if (ghost_row || ghost_col) {
            const T bv = ghost_col ? bvx : (r < 0 ? k.bcv[2] : k.bcv[3]);
            T fe[Q], fg[Q];
            feq_all(k, phi, fe);
            feq_all(k, T(2) * bv - phi, fg);
#pragma unroll
            for (int i = 0; i < Q; ++i) P[i] = fg[i] + (P[i] - fe[i]);
        }
    };
    // tangential x-slope of P (zero on ghost rows: only ever weighted by zero there)
    auto grad_x = [&](int r, const T (&P)[Q], T (&Gx)[Q]) {
        const T ig = (!a.yper && (r < 0 || r >= ny)) ? T(0) : igx_in;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            Gx[i] = T(0);
            if (EX(i) != 0) Gx[i] = (shfl_dn(P[i]) - shfl_up(P[i])) * ig;
        }
    };
    // this row's half of the y-face above it (face r+1/2, lower cell)
    auto lower_half = [&](int r, const T (&P)[Q], const T (&Gx)[Q], T (&Ly)[Q]) {
        const FaceM<T> f = a.fy[r + 2];
        const T ay[3] = {(T(1) - f.w) - f.hcd, T(1) - f.w, (T(1) - f.w) + f.hcd};
        const T g = k.hc * f.tl;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T v = ay[EY(i) + 1] * P[i];
            if (EX(i) != 0) v = fma(-T(EX(i)) * g, Gx[i], v);
            Ly[i] = v;
        }
    };
    // y-face r-1/2 from the lower half Ly and this row (upper cell): original f of the crossing velocities
    auto y_face = [&](int r, const T (&P)[Q], const T (&Gx)[Q], const T (&Ly)[Q], T (&fy)[6]) {
        const FaceM<T> f = a.fy[r + 1];
        const T ay[3] = {f.w + f.hcd, f.w, f.w - f.hcd};
        const T g = k.hc * f.tr;
        T fb[Q];
        T phib = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T v = ay[EY(i) + 1] * P[i];
            if (EX(i) != 0) v = fma(-T(EX(i)) * g, Gx[i], v);
            fb[i] = Ly[i] + v;
            phib += fb[i];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (YSLOT(i) >= 0) fy[YSLOT(i)] = fma(k.a_f, fb[i], hf_i(k, i, phib));
    };
    // x-faces of row kr and its cell update (Eq. 2.12)
    auto x_update = [&](int kr, const T (&P0)[Q], const T (&P)[Q], const T (&Pm)[6], const T (&Fp0)[Q],
                        const T (&fN)[6], const T (&fS)[6]) {
        const CellM<T> cyk = a.cy[kr + 1];
        const T igy = (ghost_col || (EDGE && role == ROLE_OUT)) ? T(0) : cyk.ig;
        T fb[Q];
        T phib = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T lx = axL[EX(i) + 1] * P0[i], rxh = axR[EX(i) + 1] * P0[i];
            if (EY(i) != 0) {
                const T gyv = (P[i] - Pm[YSLOT(i)]) * igy;
                lx = fma(-T(EY(i)) * gxL, gyv, lx);
                rxh = fma(-T(EY(i)) * gxR, gyv, rxh);
            }
            fb[i] = lx + shfl_dn(rxh);
            phib += fb[i];
        }
        T fEx[6], dW[6];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (XSLOT(i) >= 0) fEx[XSLOT(i)] = fma(k.a_f, fb[i], hf_i(k, i, phib));
#pragma unroll
        for (int o = 0; o < 6; ++o) dW[o] = fEx[o] - shfl_up(fEx[o]);  // east minus west (lane - 1's east)
        if (updates) {
            T* out = a.fout + (long long)kr * a.pitch + j;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = Fp0[i];
                if (XSLOT(i) >= 0) v = fma(-T(EX(i)) * rx, dW[XSLOT(i)], v);
                if (YSLOT(i) >= 0) v = fma(-T(EY(i)) * cyk.r, fN[YSLOT(i)] - fS[YSLOT(i)], v);
                out[i * a.plane] = v;
            }
        }
    };

    bool failed = false;
    T ft[Q], P0[Q], Fp0[Q], Pm[6], Ly[Q], fS[6], Gx[Q];
    // ---- pipeline fill: rows y0-1 and y0 ----
    if (!load_row(y0 - 1, ft)) { failed = true; }
    if (!failed) {
        cell_row(y0 - 1, ft, P0, Fp0);
        grad_x(y0 - 1, P0, Gx);
        lower_half(y0 - 1, P0, Gx, Ly);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (EY(i) != 0) Pm[YSLOT(i)] = P0[i];
        if (!load_row(y0, ft)) failed = true;
    }
    if (!failed) {
        cell_row(y0, ft, P0, Fp0);
        grad_x(y0, P0, Gx);
        y_face(y0, P0, Gx, Ly, fS);
        lower_half(y0, P0, Gx, Ly);
        // ---- steady state: row r enters, row r-1 is updated ----
#pragma unroll 2
        for (int r = y0 + 1; r <= y1; ++r) {
            T P[Q], Fp[Q], fN[6];
            if (!load_row(r, ft)) { failed = true; break; }
            cell_row(r, ft, P, Fp);
            grad_x(r, P, Gx);
            y_face(r, P, Gx, Ly, fN);
            lower_half(r, P, Gx, Ly);
            x_update(r - 1, P0, P, Pm, Fp0, fN, fS);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (EY(i) != 0) Pm[YSLOT(i)] = P0[i];
                P0[i] = P[i];
                Fp0[i] = Fp[i];
            }
#pragma unroll
            for (int o = 0; o < 6; ++o) fS[o] = fN[o];
        }
    }
    if (failed && lane == 0) {
        // record the timeout; wait (bounded) for this warp's copies still in flight
        atomicOr(a.err, 1);
        for (int q = consumed; q < issued; ++q) {
            mbar_wait_bounded(&bars[s], ph, 100000000ull);
            if (++s == S) { s = 0; ph ^= 1u; }
        }
    }
    __syncwarp();
}

template <typename T, int NC>
__global__ void __launch_bounds__(32) fused_step(const __grid_constant__ CUtensorMap tin, const StepArgs<T, NC> a,
                                                 const Consts<T, NC> k, const int seg_rows, const int S) {
    using L = WarpLayout<T>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned; the layout reserves 128 bytes of slack
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(S) * L::STAGE_BYTES);
    const int lane = threadIdx.x;
    const int xw = blockIdx.x * L::WI;
    const int y0 = blockIdx.y * seg_rows;
    const int y1 = min(y0 + seg_rows, a.ny);
    if (y0 >= a.ny || xw >= a.nx) return;
    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool edge = xw - 1 < 0 || xw + L::WI >= a.nx;
    if (edge) warp_rows<T, NC, true, false>(&tin, a, k, smem, bars, S, lane, xw, y0, y1, nullptr);
    else warp_rows<T, NC, false, false>(&tin, a, k, smem, bars, S, lane, xw, y0, y1, nullptr);
}

// the fused step with the source terms F and R (same grid and shared memory as fused_step)
template <typename T, int NC>
__global__ void __launch_bounds__(32) fused_step_src(const __grid_constant__ CUtensorMap tin, const StepArgs<T, NC> a,
                                                     const Consts<T, NC> k, const int seg_rows, const int S,
                                                     const __grid_constant__ SrcArgs<T> sa) {
    using L = WarpLayout<T>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(S) * L::STAGE_BYTES);
    const int lane = threadIdx.x;
    const int xw = blockIdx.x * L::WI;
    const int y0 = blockIdx.y * seg_rows;
    const int y1 = min(y0 + seg_rows, a.ny);
    if (y0 >= a.ny || xw >= a.nx) return;
    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool edge = xw - 1 < 0 || xw + L::WI >= a.nx;
    if (edge) warp_rows<T, NC, true, true>(&tin, a, k, smem, bars, S, lane, xw, y0, y1, &sa);
    else warp_rows<T, NC, false, true>(&tin, a, k, smem, bars, S, lane, xw, y0, y1, &sa);
}

// ---------------------------------------------------------------------------
// fused streaming kernel, single precision, velocity pairs
// ---------------------------------------------------------------------------
//
// Same dataflow and lane layout as fused_step (one cell per lane, 30 interior
// columns per warp).  The nine velocities are grouped into the opposite
// pairs q = (1,3), (2,4), (5,7), (6,8) plus the rest velocity 0; a pair is one
// float2 and runs on the packed FP32 instructions of sm_100+ (__fadd2_rn,
// __fmul2_rn, __ffma2_rn), halving the issue slots of the per-velocity
// arithmetic.  The pair's second velocity is the opposite of the first, so
// every per-pair weight has the form (a + s b, a - s b).

// pair q holds velocities (PA(q), PB(q)); QX, QY = direction of PA(q)
__host__ __device__ constexpr int PA(int q) { return q == 0 ? 1 : q == 1 ? 2 : q == 2 ? 5 : 6; }
__host__ __device__ constexpr int PB(int q) { return q == 0 ? 3 : q == 1 ? 4 : q == 2 ? 7 : 8; }
__host__ __device__ constexpr int QX(int q) { return EX(PA(q)); }
__host__ __device__ constexpr int QY(int q) { return EY(PA(q)); }

struct V9 {
    F2 p[4];
    float z;  // rest velocity
};

template <int NC>
struct ConstsP {
    float2 hbp[4][NC];  // per pair: b_bp * (feq_PA, feq_PB) coefficients in powers of phi
    float2 hf[4][NC];   // per pair: b_f * (feq_PA, feq_PB)
    float2 a_bp2, a_f2, third2;
    float a_bp, b_bp, third, hc;
    Consts<float, NC> s;  // scalar constants (ghost cells)
};

template <int NC>
__device__ __forceinline__ F2 hbp2(const ConstsP<NC>& k, int q, F2 x) {
    F2 s{k.hbp[q][NC - 1]};
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma2(s, x, F2{k.hbp[q][m]});
    return s;
}
template <int NC>
__device__ __forceinline__ F2 hf2(const ConstsP<NC>& k, int q, F2 x) {
    F2 s{k.hf[q][NC - 1]};
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma2(s, x, F2{k.hf[q][m]});
    return s;
}
__device__ __forceinline__ float vsum(const V9& a) {
    const F2 s = (a.p[0] + a.p[1]) + (a.p[2] + a.p[3]);
    return a.z + (s.v.x + s.v.y);
}

// Source terms of one cell added to the velocity pairs of P and Fp (the
// arithmetic of add_source on the scalar path, with phi^n and phi^{n-1} carried
// as one pair).  Av[0..7] are the cell's field values S_k, in ascending order of
// power, and Av[8] its phi^{n-1}, staged with its ftilde.  Each pair holds two
// opposite velocities, so their c_i.u terms differ only in sign and their
// weights agree.  The loops run to fixed bounds: the host leaves en, ep and
// dpow of the unused terms and the b' coefficients beyond its degree at zero
// (an unused term reads a valid field and weighs it by zero), so no branch
// depends on the number of terms.  b has degree <= NC - 1 wherever B = u b(phi)
// enters the equilibrium; with u = 0 the R terms vanish whatever b' is.
template <int NC>
__device__ __forceinline__ void add_source_vp(const SrcArgs<float>& sa, const float (&Av)[9], float phi, V9& P,
                                              V9& Fp) {
    const F2 X = f2(phi, sa.first ? phi : Av[8]);  // (phi^n, phi^{n-1})
    F2 pw = f2(1.f), Fs = f2(0.f);                 // X^power[k]; (F^n, F^{n-1})
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        for (int m = 0; m < sa.dpow[q]; ++m) pw = pw * X;
        Fs = fma2(f2(sa.en[q], sa.ep[q]) * f2(Av[q]), pw, Fs);
    }
    F2 d = f2(0.f);  // (b'(phi^n), b'(phi^{n-1}))
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) d = fma2(d, X, f2(sa.db[m]));
    const F2 G = d * Fs;  // (g^n, g^{n-1}) = b' F
    // F and g at the interface (backward difference over dt/2) and at the update
    const float Ft = fmaf(0.25f, Fs.v.x - Fs.v.y, Fs.v.x), gt = fmaf(0.25f, G.v.x - G.v.y, G.v.x);
    const float Fa = fmaf(0.5f, Fs.v.x - Fs.v.y, Fs.v.x), ga = fmaf(0.5f, G.v.x - G.v.y, G.v.x);
    const F2 gt2 = f2(gt), ga2 = f2(ga);
    const F2 aP1 = f2(sa.kP_f[1] * Ft), aP2 = f2(sa.kP_f[5] * Ft);  // weight 1/9 and 1/36 pairs
    const F2 aU1 = f2(sa.kU_f[1] * Fa), aU2 = f2(sa.kU_f[5] * Fa);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        P.p[q] = P.p[q] + fma2(f2(sa.kP_g[PA(q)], sa.kP_g[PB(q)]), gt2, q < 2 ? aP1 : aP2);
        Fp.p[q] = Fp.p[q] + fma2(f2(sa.kU_g[PA(q)], sa.kU_g[PB(q)]), ga2, q < 2 ? aU1 : aU2);
    }
    P.z = fmaf(sa.kP_f[0], Ft, P.z);  // the rest velocity has c_0 = 0
    Fp.z = fmaf(sa.kU_f[0], Fa, Fp.z);
}

// One warp waits, bounded, on an mbarrier that nothing completes: the wait expires and the
// error word is set, as after a stalled copy in a step kernel.
__global__ void __launch_bounds__(32) wait_timeout_kernel(int* err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (__any_sync(0xffffffffu, !ok) && threadIdx.x == 0) atomicOr(err, 1);
}

// ---------------------------------------------------------------------------
// initialisation and moments
// ---------------------------------------------------------------------------

// ftilde_i = feq_i(phi0) (opening of Section 4).  phi0 is [ny][nx] contiguous.  With err
// set, an equilibrium negative by more than 1e-3 of the cell's largest one (Eq. 2.3 allows
// it for large |B|/c or D) sets bit 2 (value 4) of the error word.
template <typename T, int NC, typename Tin>
__global__ void init_kernel(const Tin* __restrict__ phi0, T* __restrict__ f, int nx, int ny, long long pitch,
                            long long plane, const Consts<T, NC> k, int* err) {
    const long long n = (long long)nx * ny;
    bool neg = false;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int kr = int(c / nx), j = int(c % nx);
        T fe[Q];
        feq_all(k, T(phi0[c]), fe);
        T mn = fe[0], mx = fabs(fe[0]);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i * plane + kr * pitch + j] = fe[i];
            mn = fmin(mn, fe[i]);
            mx = fmax(mx, fabs(fe[i]));
        }
        neg |= mn + T(1e-3) * mx < T(0);
    }
    if (neg && err) atomicOr(err, 4);
}

// phi = sum_i ftilde_i (optionally stored as Tout), and per-block partial
// sums of |V| phi in double.  Blocks of 256 threads.
template <typename T, typename Tout>
__global__ void __launch_bounds__(256) phi_mass_kernel(const T* __restrict__ f, Tout* __restrict__ phi, int nx, int ny,
                                                       long long pitch, long long plane, const double* __restrict__ dxv,
                                                       const double* __restrict__ dyv, double* __restrict__ partial) {
    const long long n = (long long)nx * ny;
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int kr = int(c / nx), j = int(c % nx);
        T s = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) s += f[i * plane + kr * pitch + j];
        if (phi) phi[c] = Tout(s);
        acc += dxv[j] * dyv[kr] * double(s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += ws[w];
        partial[blockIdx.x] = s;
    }
}

// Sum of the block partials in a fixed order (deterministic), one block of 256.
__global__ void __launch_bounds__(256) sum_partials_kernel(const double* __restrict__ partial, int n,
                                                           double* __restrict__ out) {
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
        *out = s;
    }
}

}  // namespace dugks

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

template <typename T, int NC, bool EDGE>
__device__ __forceinline__ void warp_rows(const CUtensorMap* tin, const StepArgs<T, NC>& a, const Consts<T, NC>& k,
                                          unsigned char* stages, uint64_t* bars, const int S, const int lane,
                                          const int xw, const int y0, const int y1) {
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
    const int soff = scol - xs;  // this lane's column inside a stage row

    // per-lane x-face coefficients: value weights for e_x = -1, 0, +1 and the tangential weights
    T axL[3], axR[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        axL[e] = (T(1) - fE.w) + T(e - 1) * fE.hcd;  // this cell as the left cell of its east face
        axR[e] = fW.w - T(e - 1) * fW.hcd;           // this cell as the right cell of its west face
    }
    const T gxL = k.hc * fE.tl, gxR = k.hc * fW.tr;

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

    T P0[Q], Pm[6], Fp0[Q], Ly[Q], fS[6];
#pragma unroll
    for (int i = 0; i < Q; ++i) { P0[i] = T(0); Fp0[i] = T(0); Ly[i] = T(0); }
#pragma unroll
    for (int o = 0; o < 6; ++o) { Pm[o] = T(0); fS[o] = T(0); }

    int s = 0;
    uint32_t ph = 0;
    int idx = 0;
    bool failed = false;
    for (; idx < R; ++idx) {
        const int r = y0 - 1 + idx;
        const bool ok = mbar_wait_bounded(&bars[s], ph, 2000000000ull);
        if (__any_sync(0xffffffffu, !ok)) { failed = true; break; }
        // ---- P (and Fp) of row r for this lane's column ----
        const T* st = reinterpret_cast<const T*>(stages + size_t(s) * L::STAGE_BYTES);
        T ft[Q];
        if (from_smem) {
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = st[i * L::BOXW + soff];
        } else if (role != ROLE_OUT) {
            const int sr = src_row(r);
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = a.fin[i * a.plane + (long long)sr * a.pitch + scol];
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = T(0);
        }
        __syncwarp();
        if (lane == 0 && idx + S < R) {  // refill the stage just consumed
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[s], uint32_t(L::BOX_BYTES));
            tma_load_3d(stages + size_t(s) * L::STAGE_BYTES, tin, &bars[s], xs, src_row(r + S), 0);
        }
        if (++s == S) { s = 0; ph ^= 1u; }
        T phi = ft[0];
#pragma unroll
        for (int i = 1; i < Q; ++i) phi += ft[i];
        T fe[Q], P[Q], Fp[Q];
        feq_all(k, phi, fe);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            P[i] = fma(k.a_bp, ft[i], k.b_bp * fe[i]);
            Fp[i] = fma(k.a_tp, ft[i], k.b_tp * fe[i]);
        }
        const bool ghost_row = !a.yper && (r < 0 || r >= ny);
        if (ghost_row || ghost_col) {
            const T bv = ghost_col ? bvx : (r < 0 ? k.bcv[2] : k.bcv[3]);
            T fg[Q];
            feq_all(k, T(2) * bv - phi, fg);
#pragma unroll
            for (int i = 0; i < Q; ++i) P[i] = fg[i] + (P[i] - fe[i]);
        }
        // ---- tangential x-slope of row r, y-face r-1/2 and the lower half of r+1/2 ----
        const FaceM<T> fyR = a.fy[r + 1], fyN = a.fy[r + 2];
        const T igx = ghost_row ? T(0) : cxj.ig;
        T Gx[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            Gx[i] = T(0);
            if (EX(i) != 0) Gx[i] = (shfl_dn(P[i]) - shfl_up(P[i])) * igx;
        }
        T fN[6];
        if (idx >= 1) {
            const T ayR[3] = {fyR.w + fyR.hcd, fyR.w, fyR.w - fyR.hcd};
            const T gy = k.hc * fyR.tr;
            T fb[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = ayR[EY(i) + 1] * P[i];
                if (EX(i) != 0) v = fma(-T(EX(i)) * gy, Gx[i], v);
                fb[i] = Ly[i] + v;
            }
            face_original<T, NC, false>(k, fb, fN);
        }
        {
            const T ayL[3] = {(T(1) - fyN.w) - fyN.hcd, T(1) - fyN.w, (T(1) - fyN.w) + fyN.hcd};
            const T gy = k.hc * fyN.tl;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T v = ayL[EY(i) + 1] * P[i];
                if (EX(i) != 0) v = fma(-T(EX(i)) * gy, Gx[i], v);
                Ly[i] = v;
            }
        }
        // ---- x-faces and update of row kr = r-1 ----
        if (idx >= 2) {
            const int kr = r - 1;
            const CellM<T> cyk = a.cy[kr + 1];
            const T igy = ghost_col || (EDGE && role == ROLE_OUT) ? T(0) : cyk.ig;
            T fb[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T lx = axL[EX(i) + 1] * P0[i], rx = axR[EX(i) + 1] * P0[i];
                if (EY(i) != 0) {
                    const T gyv = (P[i] - Pm[YSLOT(i)]) * igy;
                    lx = fma(-T(EY(i)) * gxL, gyv, lx);
                    rx = fma(-T(EY(i)) * gxR, gyv, rx);
                }
                fb[i] = lx + shfl_dn(rx);
            }
            T fEx[6], fWx[6];
            face_original<T, NC, true>(k, fb, fEx);
#pragma unroll
            for (int o = 0; o < 6; ++o) fWx[o] = shfl_up(fEx[o]);  // west face = east face of lane - 1
            if (updates) {
                T* out = a.fout + (long long)kr * a.pitch + j;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    T v = Fp0[i];
                    if (XSLOT(i) >= 0) v = fma(-T(EX(i)) * cxj.r, fEx[XSLOT(i)] - fWx[XSLOT(i)], v);
                    if (YSLOT(i) >= 0) v = fma(-T(EY(i)) * cyk.r, fN[YSLOT(i)] - fS[YSLOT(i)], v);
                    out[i * a.plane] = v;
                }
            }
        }
        // ---- rotate the row window ----
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (EY(i) != 0) Pm[YSLOT(i)] = P0[i];
            P0[i] = P[i];
            Fp0[i] = Fp[i];
        }
        if (idx >= 1) {
#pragma unroll
            for (int o = 0; o < 6; ++o) fS[o] = fN[o];
        }
    }
    if (failed && lane == 0) {
        // record the timeout; wait (bounded) for this warp's copies still in flight
        atomicOr(a.err, 1);
        for (int q = idx; q < min(idx + S, R); ++q) {
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
    if (edge) warp_rows<T, NC, true>(&tin, a, k, smem, bars, S, lane, xw, y0, y1);
    else warp_rows<T, NC, false>(&tin, a, k, smem, bars, S, lane, xw, y0, y1);
}

// ---------------------------------------------------------------------------
// initialisation and moments
// ---------------------------------------------------------------------------

// ftilde_i = feq_i(phi0) (opening of Section 4).  phi0 is [ny][nx] contiguous.
template <typename T, int NC, typename Tin>
__global__ void init_kernel(const Tin* __restrict__ phi0, T* __restrict__ f, int nx, int ny, long long pitch,
                            long long plane, const Consts<T, NC> k) {
    const long long n = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int kr = int(c / nx), j = int(c % nx);
        T fe[Q];
        feq_all(k, T(phi0[c]), fe);
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i * plane + kr * pitch + j] = fe[i];
    }
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

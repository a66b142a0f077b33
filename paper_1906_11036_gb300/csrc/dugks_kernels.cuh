// dugks_kernels.cuh -- the DUGKS step kernels (arXiv:1906.11036, Section 2,
// step summary at the end of the section), plus initialisation and the
// phi / mass reduction.
//
//   naive_step  : one thread per cell; recomputes P = fbar^+ of its 3x3
//                 neighbourhood straight from global memory.  A simple
//                 cross-check of the fused kernel.
//   fused_step  : the production kernel.  A CTA owns a strip of NT-2
//                 columns (plus one halo column on each side) and a segment
//                 of rows, and marches up the segment one row at a time.
//                 Each row of ftilde (all nine planes) arrives in shared
//                 memory by one 3-D TMA copy, several rows ahead, so ftilde
//                 is read once and written once per step.  P of the last
//                 three rows, the y-face flux of the row below and the lower
//                 half of the next y-face stay in registers; x-neighbours
//                 exchange their halves of the x-face through shared memory.
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

template <typename T, int NT>
struct FusedLayout {
    static constexpr int ALIGN = 16 / int(sizeof(T));  // TMA x-coordinate granule (16 bytes)
    static constexpr int BOXW = NT + ALIGN;            // columns per TMA box row
    static constexpr int STAGE_BYTES = ((Q * BOXW * int(sizeof(T)) + 127) / 128) * 128;
    static constexpr int PROW = NT + 2;
    static constexpr int XROW = NT + 1;
    static size_t bytes(int stages) {
        return size_t(stages) * STAGE_BYTES + size_t(stages) * 8 +
               sizeof(T) * (size_t(Q) * PROW + size_t(Q) * XROW + size_t(6) * XROW) + 128;
    }
};

enum ColRole { ROLE_IN = 0, ROLE_GHOST_W, ROLE_GHOST_E, ROLE_WRAP_W, ROLE_WRAP_E, ROLE_OUT };

template <typename T, int NC, int NT>
__global__ void __launch_bounds__(NT) fused_step(const __grid_constant__ CUtensorMap tin, const StepArgs<T, NC> a,
                                                 const Consts<T, NC> k, const int seg_rows, const int S) {
    using L = FusedLayout<T, NT>;
    constexpr int W = NT - 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned; the layout reserves 128 bytes of slack
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    unsigned char* stage_base = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(S) * L::STAGE_BYTES);
    T* Prow = reinterpret_cast<T*>(bars + S);  // [Q][PROW]
    T* RX = Prow + Q * L::PROW;                // [Q][XROW]
    T* FX = RX + Q * L::XROW;                  // [6][XROW]

    const int t = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int x0 = blockIdx.x * W;
    const int j = x0 - 1 + t;
    const int xs = (x0 - 1) & ~(L::ALIGN - 1);
    const int y0 = blockIdx.y * seg_rows;
    const int y1 = min(y0 + seg_rows, ny);
    if (y0 >= ny) return;
    const int R = y1 - y0 + 2;  // rows r = y0-1 .. y1 pass through the pipeline

    int role, scol;
    if (j >= 0 && j < nx) { role = ROLE_IN; scol = j; }
    else if (j == -1) { role = a.xper ? ROLE_WRAP_W : ROLE_GHOST_W; scol = a.xper ? nx - 1 : 0; }
    else if (j == nx) { role = a.xper ? ROLE_WRAP_E : ROLE_GHOST_E; scol = a.xper ? 0 : nx - 1; }
    else { role = ROLE_OUT; scol = 0; }
    const bool from_smem = role == ROLE_IN || role == ROLE_GHOST_W || role == ROLE_GHOST_E;
    const bool updates = role == ROLE_IN && t >= 1 && t <= W;
    const bool ghost_col = role == ROLE_GHOST_W || role == ROLE_GHOST_E;
    const int jm = min(max(j, -1), nx);  // clamped index for metric loads
    const FaceM<T> fW = a.fx[jm + 1], fE = a.fx[jm + 2];
    const CellM<T> cxj = a.cx[jm + 1];
    const T bvx = role == ROLE_GHOST_W ? k.bcv[0] : k.bcv[1];

    if (t == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto src_row = [&](int r) -> int {
        if (r >= 0 && r < ny) return r;
        if (a.yper) return ((r % ny) + ny) % ny;
        return r < 0 ? 0 : ny - 1;
    };
    auto issue = [&](int idx) {
        const int s = idx % S;
        unsigned char* dst = stage_base + size_t(s) * L::STAGE_BYTES;
        mbar_arrive_expect_tx(&bars[s], uint32_t(Q * L::BOXW * sizeof(T)));
        tma_load_3d(dst, &tin, &bars[s], xs, src_row(y0 - 1 + idx), 0);
    };
    if (t == 0) {
        for (int idx = 0; idx < min(S, R); ++idx) issue(idx);
    }

    T P0[Q], Pm[6], Fp0[Q], Ly[Q], fS[6];
#pragma unroll
    for (int i = 0; i < Q; ++i) { P0[i] = T(0); Fp0[i] = T(0); Ly[i] = T(0); }
#pragma unroll
    for (int o = 0; o < 6; ++o) { Pm[o] = T(0); fS[o] = T(0); }

    int idx = 0;
    bool failed = false;
    for (; idx < R; ++idx) {
        const int r = y0 - 1 + idx;
        const int s = idx % S;
        const bool ok = mbar_wait_bounded(&bars[s], uint32_t((idx / S) & 1), 2000000000ull);
        // ---- P (and Fp) of row r for this thread's column ----
        const T* st = reinterpret_cast<const T*>(stage_base + size_t(s) * L::STAGE_BYTES);
        const int sr = src_row(r);
        T ft[Q], fe[Q], P[Q], Fp[Q];
        T phi = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T v = T(0);
            if (from_smem) v = st[i * L::BOXW + (scol - xs)];
            else if (role != ROLE_OUT) v = a.fin[i * a.plane + sr * a.pitch + scol];
            ft[i] = v;
            phi += v;
        }
        feq_all(k, phi, fe);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            P[i] = fma(k.a_bp, ft[i], k.b_bp * fe[i]);
            Fp[i] = fma(k.a_tp, ft[i], k.b_tp * fe[i]);
        }
        const bool ghost_row = !a.yper && (r < 0 || r >= ny);
        if (ghost_col || ghost_row) {
            const T bv = ghost_col ? bvx : (r < 0 ? k.bcv[2] : k.bcv[3]);
            T fg[Q];
            feq_all(k, T(2) * bv - phi, fg);
#pragma unroll
            for (int i = 0; i < Q; ++i) P[i] = fg[i] + (P[i] - fe[i]);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) Prow[i * L::PROW + t + 1] = P[i];
        const int bad = __syncthreads_or(ok ? 0 : 1);
        if (bad) { failed = true; break; }
        if (t == 0 && idx + S < R) {
            fence_proxy_async_smem();
            issue(idx + S);
        }
        // ---- y-face r-1/2 (lower half carried in Ly) and upper half for r+1/2 ----
        T Gx[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) Gx[i] = T(0);
        if (updates && !ghost_row) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (EX(i) != 0) Gx[i] = (Prow[i * L::PROW + t + 2] - Prow[i * L::PROW + t]) * cxj.ig;
        }
        const FaceM<T> fyR = a.fy[r + 1], fyN = a.fy[r + 2];
        T fN[6];
        if (idx >= 1) {
            T fb[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i)
                fb[i] = Ly[i] + ((fyR.w - T(EY(i)) * fyR.hcd) * P[i] - T(EX(i)) * k.hc * fyR.tr * Gx[i]);
            face_original<T, NC, false>(k, fb, fN);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i)
            Ly[i] = ((T(1) - fyN.w) + T(EY(i)) * fyN.hcd) * P[i] - T(EX(i)) * k.hc * fyN.tl * Gx[i];
        // ---- x-faces and update of row k = r-1 ----
        if (idx >= 2) {
            const int kr = r - 1;
            const CellM<T> cyk = a.cy[kr + 1];
            T Gy[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) Gy[i] = T(0);
            if (!ghost_col && role != ROLE_OUT) {
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if (EY(i) != 0) Gy[i] = (P[i] - Pm[YSLOT(i)]) * cyk.ig;
            }
            T Lx[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                Lx[i] = ((T(1) - fE.w) + T(EX(i)) * fE.hcd) * P0[i] - T(EY(i)) * k.hc * fE.tl * Gy[i];
                RX[i * L::XROW + t] = (fW.w - T(EX(i)) * fW.hcd) * P0[i] - T(EY(i)) * k.hc * fW.tr * Gy[i];
            }
            __syncthreads();
            T fb[Q], fEx[6];
#pragma unroll
            for (int i = 0; i < Q; ++i) fb[i] = Lx[i] + RX[i * L::XROW + t + 1];
            face_original<T, NC, true>(k, fb, fEx);
#pragma unroll
            for (int o = 0; o < 6; ++o) FX[o * L::XROW + t] = fEx[o];
            __syncthreads();
            if (updates) {
                T* out = a.fout + (long long)kr * a.pitch + j;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    T v = Fp0[i];
                    if (XSLOT(i) >= 0)
                        v -= T(EX(i)) * cxj.r * (fEx[XSLOT(i)] - FX[XSLOT(i) * L::XROW + t - 1]);
                    if (YSLOT(i) >= 0) v -= T(EY(i)) * cyk.r * (fN[YSLOT(i)] - fS[YSLOT(i)]);
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
    if (failed) {
        // record the timeout and wait (bounded) for this CTA's copies still in flight
        if (t == 0) {
            atomicOr(a.err, 1);
            for (int q = idx; q < min(idx + S, R); ++q) mbar_wait_bounded(&bars[q % S], uint32_t((q / S) & 1), 100000000ull);
        }
        __syncthreads();
    }
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

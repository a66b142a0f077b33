// dugks3d_kernels.cuh -- the DUGKS step of Section 2 (arXiv:1906.11036) in
// three dimensions with the D3Q15 (Eq. 2.28) or D3Q19 (Eq. 2.6) velocity set.
//
// step3d: one CTA of NW warps owns a tile of 30 columns (lanes 1..30 of each
// warp; lanes 0 and 31 hold the x-halo) by NW-2 rows (warps 1..NW-2; warps 0
// and NW-1 hold the y-halo) and marches up a segment of z-planes.  For every
// plane it computes P = fbar^+ (Eq. 2.21) of all its cells into a three-plane
// shared-memory ring, then each interior cell builds three faces from the ring:
// its east x-face, its north y-face and its top z-face (Eqs. 2.19, 2.20, 2.26,
// phi_b, Eq. 2.22).  The west x-face arrives from the lane to the left by a
// warp shuffle, the south y-face from the row below through shared memory, and
// the bottom z-face is the top face of the plane below, kept in registers.
// The update (Eq. 2.12) reads ftilde of the cell again (an L1/L2 hit) to form
// ftilde^+ = P + (P - ftilde)/3 (Eq. 2.23).
//
// ftilde of the planes is staged with cp.async into a three-plane ring of
// per-thread shared-memory slots beside the P ring: while plane z is
// processed, ftilde(z) waits for the update, ftilde(z+1) feeds P and
// ftilde(z+2) is in flight.  A thread only touches its own slots, and refills a
// slot only after its own update has read it.
//
// Only the velocities that cross a face need their reconstructed fbar; the
// interface phi_b = sum_i fbar_i follows from the moments M0 = sum_i P_i and
// M_a = sum_i e_a P_i of the two cells (the reconstruction is linear):
//   phi_b = (1-w) M0_L + w M0_R + hcd (Mn_L - Mn_R)
//           - hc [tl sum_t d_t M_t (L) + tr sum_t d_t M_t (R)]
// with d_t the same central differences along the tangential axes t.  Each
// cell stores its four moments next to P.
//
// Halo cells (periodic images, mirrored Dirichlet ghosts, or cells beyond the
// domain) take their ftilde from the wrapped or clamped interior cell; a ghost
// applies the non-equilibrium extrapolation P_g = feq(2 bv - phi) + P - feq(phi).
// Cells beyond the domain only ever meet zero weights.
#pragma once
#include <cuda.h>

#include "dugks_device.cuh"

namespace dugks3 {

using dugks::CellM;
using dugks::FaceM;

// Direction components in units of c, rows x, y, z ('+' = 1, '-' = -1):
// D3Q19 as Eq. 2.6 lists them, D3Q15 as Eq. 2.28.
template <int QQ>
__host__ __device__ constexpr char D3CH(int i, int a) {
    return (QQ == 19 ? "0+-0000+-+-+--+0000"
                       "000+-00+--+0000+-+-"
                       "00000+-0000+-+-+--+"
                     : "0+-0000+++----+"
                       "000+-00++-+--+-"
                       "00000+-+-++-+--")[a * QQ + i];
}
template <int QQ>
__host__ __device__ constexpr int E3(int i, int a) {
    return D3CH<QQ>(i, a) == '+' ? 1 : (D3CH<QQ>(i, a) == '-' ? -1 : 0);
}

// position of velocity i among those that cross a face normal to axis a (-1: parallel)
template <int QQ>
__host__ __device__ constexpr int XS3(int i, int a) {
    if (E3<QQ>(i, a) == 0) return -1;
    int s = 0;
    for (int m = 0; m < i; ++m) s += E3<QQ>(m, a) != 0 ? 1 : 0;
    return s;
}

constexpr int NCROSS = 10;  // velocities crossing a face of either lattice

static_assert(E3<19>(11, 0) == 1 && E3<19>(11, 2) == 1 && E3<19>(17, 1) == 1 && E3<19>(17, 2) == -1, "D3Q19 table");
static_assert(E3<15>(13, 0) == -1 && E3<15>(13, 1) == 1 && E3<15>(13, 2) == -1, "D3Q15 table");
static_assert(XS3<19>(18, 2) == NCROSS - 1 && XS3<15>(14, 0) == NCROSS - 1, "crossing counts");

template <typename T, int QQ, int NC>
struct Consts3 {
    T feq[QQ][NC];  // feq_i(phi) = sum_m feq[i][m] phi^m (ghosts)
    T hbp[QQ][NC];  // b_bp feq[i][m]: P = a_bp ft + hbp_i(phi)
    T hf[QQ][NC];   // b_f feq[i][m]: f = a_f fbar + hf_i(phi_b)
    T a_bp, b_bp, a_f, third, hc;
    T bcv[6];       // Dirichlet wall values W, E, S, N, B, T
};

template <typename T>
struct Args3 {
    const T* fin;
    T* fout;
    int nx, ny, nz;
    long long plane;        // nx ny nz: elements per velocity, layout [Q][nz][ny][nx]
    int per[3];             // periodic flags per axis
    const FaceM<T>* fm[3];  // per axis, faces f = -1 .. n+1 at index f+1
    const CellM<T>* cm[3];  // per axis, cells j = -1 .. n at index j+1
    int zseg;               // planes per CTA segment
    int* err;               // device error word: bit 0 = a bounded TMA wait expired
};

template <typename T, int QQ, int NC>
__device__ __forceinline__ T horner3(const T (&c)[QQ][NC], int i, T x) {
    T s = c[i][NC - 1];
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma(s, x, c[i][m]);
    return s;
}

// periodic wrap, or clamp into the domain
__device__ __forceinline__ int wrapc(int j, int n, int per) {
    if (per) {
        j %= n;
        return j < 0 ? j + n : j;
    }
    return min(max(j, 0), n - 1);
}

template <typename T, int QQ, int NC, int NW>
__global__ void __launch_bounds__(NW * 32, 1) step3d(const Args3<T> a, const Consts3<T, QQ, NC> k) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sP = reinterpret_cast<T*>(smem_raw);  // [3][NW][QQ][32]: P of three planes
    T* sY = sP + 3 * NW * QQ * 32;           // [NW][NCROSS][32]: north y-face f of each row
    T* sM = sY + NW * NCROSS * 32;           // [3][NW][4][32]: moments M0, Mx, My, Mz of P
    T* sF = sM + 3 * NW * 4 * 32;            // [3][NW][QQ][32]: ftilde of three planes (cp.async)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x0 = blockIdx.x * 30, y0 = blockIdx.y * (NW - 2), z0 = blockIdx.z * a.zseg;
    if (z0 >= a.nz) return;  // uniform over the CTA
    const int z1 = min(z0 + a.zseg, a.nz);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int j = x0 - 1 + lane, kk = y0 - 1 + w;
    const int sj = wrapc(j, nx, a.per[0]), sk = wrapc(kk, ny, a.per[1]);
    const bool gx = !a.per[0] && (j < 0 || j >= nx), gy = !a.per[1] && (kk < 0 || kk >= ny);
    const int jm = min(max(j, -1), nx), km = min(max(kk, -1), ny);
    const FaceM<T> fE = a.fm[0][jm + 2], fN = a.fm[1][km + 2];
    const CellM<T> cxj = a.cm[0][jm + 1], cyk = a.cm[1][km + 1];
    const bool interior_row = w >= 1 && w <= NW - 2;
    const bool interior_col = lane >= 1 && lane <= 30;
    const bool updates = interior_row && interior_col && j < nx && kk < ny;

    auto Ps = [&](int slot, int ww, int i, int l) -> T { return sP[((slot * NW + ww) * QQ + i) * 32 + l]; };
    auto Ms = [&](int slot, int ww, int m, int l) -> T { return sM[((slot * NW + ww) * 4 + m) * 32 + l]; };

    // ring slot of plane zz (z0-1 <= zz <= z1+1), shared by sP, sM and sF
    auto slot_of = [&](int zz) { return (zz - z0 + 1) % 3; };
    auto Fs = [&](int slot, int i) -> T { return sF[((slot * NW + w) * QQ + i) * 32 + lane]; };
    // start the copy of this thread's ftilde of plane zz into its slots of sF
    auto prefetch = [&](int zz) {
        const long long c = ((long long)wrapc(zz, nz, a.per[2]) * ny + sk) * nx + sj;
        const int sl = slot_of(zz);
#pragma unroll
        for (int i = 0; i < QQ; ++i) {
            const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(sF + ((sl * NW + w) * QQ + i) * 32 + lane));
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(a.fin + i * a.plane + c),
                         "n"(int(sizeof(T))));
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    // P of plane zz (already prefetched into sF) into ring slot `slot`; then prefetch plane `next`
    auto compute_P = [&](int zz, int slot, int next) {
        const bool gz = !a.per[2] && (zz < 0 || zz >= nz);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        T f[QQ];
        T phi = T(0);
#pragma unroll
        for (int i = 0; i < QQ; ++i) {
            f[i] = Fs(slot, i);
            phi += f[i];
        }
        // the slot of plane next held plane next-3, whose update this thread has done
        prefetch(next);
        T P[QQ];
        T hs = T(0);
#pragma unroll
        for (int i = 1; i < QQ; ++i) {
            const T h = horner3(k.hbp, i, phi);
            P[i] = fma(k.a_bp, f[i], h);
            hs += h;
        }
        P[0] = fma(k.a_bp, f[0], fma(k.b_bp, phi, -hs));  // rest velocity via the zeroth moment
        if (gx || gy || gz) {  // mirrored ghost: P_g = feq(2 bv - phi) + P - feq(phi)
            const T bv = gx ? (j < 0 ? k.bcv[0] : k.bcv[1])
                            : (gy ? (kk < 0 ? k.bcv[2] : k.bcv[3]) : (zz < 0 ? k.bcv[4] : k.bcv[5]));
            const T pg = T(2) * bv - phi;
#pragma unroll
            for (int i = 0; i < QQ; ++i) P[i] += horner3(k.feq, i, pg) - horner3(k.feq, i, phi);
        }
        T m0 = T(0), mx = T(0), my = T(0), mz = T(0);
#pragma unroll
        for (int i = 0; i < QQ; ++i) {
            sP[((slot * NW + w) * QQ + i) * 32 + lane] = P[i];
            m0 += P[i];
            if (E3<QQ>(i, 0) != 0) mx += T(E3<QQ>(i, 0)) * P[i];
            if (E3<QQ>(i, 1) != 0) my += T(E3<QQ>(i, 1)) * P[i];
            if (E3<QQ>(i, 2) != 0) mz += T(E3<QQ>(i, 2)) * P[i];
        }
        T* M = sM + (slot * NW + w) * 4 * 32 + lane;
        M[0] = m0;
        M[32] = mx;
        M[64] = my;
        M[96] = mz;
    };

    // f of the velocities crossing the z-face between ring slots lo (below) and hi (above)
    auto z_face = [&](int lo, int hi, const FaceM<T>& fz, T (&out)[NCROSS]) {
        const int l1 = max(lane - 1, 0), l2 = min(lane + 1, 31);
        const int w1 = max(w - 1, 0), w2 = min(w + 1, NW - 1);
        const T phib = (T(1) - fz.w) * Ms(lo, w, 0, lane) + fz.w * Ms(hi, w, 0, lane) +
                       fz.hcd * (Ms(lo, w, 3, lane) - Ms(hi, w, 3, lane)) -
                       k.hc * (fz.tl * ((Ms(lo, w, 1, l2) - Ms(lo, w, 1, l1)) * cxj.ig +
                                        (Ms(lo, w2, 2, lane) - Ms(lo, w1, 2, lane)) * cyk.ig) +
                               fz.tr * ((Ms(hi, w, 1, l2) - Ms(hi, w, 1, l1)) * cxj.ig +
                                        (Ms(hi, w2, 2, lane) - Ms(hi, w1, 2, lane)) * cyk.ig));
#pragma unroll
        for (int i = 0; i < QQ; ++i) {
            if (XS3<QQ>(i, 2) < 0) continue;
            const int en = E3<QQ>(i, 2), ex = E3<QQ>(i, 0), ey = E3<QQ>(i, 1);
            T v = ((T(1) - fz.w) + T(en) * fz.hcd) * Ps(lo, w, i, lane) + (fz.w - T(en) * fz.hcd) * Ps(hi, w, i, lane);
            if (ex != 0) {
                const T gl = (Ps(lo, w, i, l2) - Ps(lo, w, i, l1)) * cxj.ig;
                const T gr = (Ps(hi, w, i, l2) - Ps(hi, w, i, l1)) * cxj.ig;
                v -= T(ex) * k.hc * (fz.tl * gl + fz.tr * gr);
            }
            if (ey != 0) {
                const T gl = (Ps(lo, w2, i, lane) - Ps(lo, w1, i, lane)) * cyk.ig;
                const T gr = (Ps(hi, w2, i, lane) - Ps(hi, w1, i, lane)) * cyk.ig;
                v -= T(ey) * k.hc * (fz.tl * gl + fz.tr * gr);
            }
            out[XS3<QQ>(i, 2)] = fma(k.a_f, v, horner3(k.hf, i, phib));
        }
    };

    // pipeline fill: planes z0-1 and z0, and the bottom face of plane z0
    prefetch(z0 - 1);
    compute_P(z0 - 1, 0, z0);
    compute_P(z0, 1, z0 + 1);
    __syncthreads();
    T fB[NCROSS];
    if (interior_row) z_face(0, 1, a.fm[2][z0 + 1], fB);

    for (int z = z0; z < z1; ++z) {
        const int sm = (z - z0) % 3, so = (z - z0 + 1) % 3, sp = (z - z0 + 2) % 3;
        compute_P(z + 1, sp, z + 2);
        __syncthreads();
        const CellM<T> czl = a.cm[2][z + 1];
        const int l1 = max(lane - 1, 0), l2 = min(lane + 1, 31);
        const int w1 = max(w - 1, 0), w2 = min(w + 1, NW - 1);
        // east x-face (lanes 0..30 of the interior rows)
        T fEx[NCROSS], fNy[NCROSS], fTz[NCROSS];
#pragma unroll
        for (int s = 0; s < NCROSS; ++s) fEx[s] = fNy[s] = fTz[s] = T(0);
        if (interior_row && lane <= 30) {
            const int lr = lane + 1;
            const T phib = (T(1) - fE.w) * Ms(so, w, 0, lane) + fE.w * Ms(so, w, 0, lr) +
                           fE.hcd * (Ms(so, w, 1, lane) - Ms(so, w, 1, lr)) -
                           k.hc * (fE.tl * ((Ms(so, w2, 2, lane) - Ms(so, w1, 2, lane)) * cyk.ig +
                                            (Ms(sp, w, 3, lane) - Ms(sm, w, 3, lane)) * czl.ig) +
                                   fE.tr * ((Ms(so, w2, 2, lr) - Ms(so, w1, 2, lr)) * cyk.ig +
                                            (Ms(sp, w, 3, lr) - Ms(sm, w, 3, lr)) * czl.ig));
#pragma unroll
            for (int i = 0; i < QQ; ++i) {
                if (XS3<QQ>(i, 0) < 0) continue;
                const int en = E3<QQ>(i, 0), ey = E3<QQ>(i, 1), ez = E3<QQ>(i, 2);
                T v = ((T(1) - fE.w) + T(en) * fE.hcd) * Ps(so, w, i, lane) + (fE.w - T(en) * fE.hcd) * Ps(so, w, i, lr);
                if (ey != 0) {
                    const T gl = (Ps(so, w2, i, lane) - Ps(so, w1, i, lane)) * cyk.ig;
                    const T gr = (Ps(so, w2, i, lr) - Ps(so, w1, i, lr)) * cyk.ig;
                    v -= T(ey) * k.hc * (fE.tl * gl + fE.tr * gr);
                }
                if (ez != 0) {
                    const T gl = (Ps(sp, w, i, lane) - Ps(sm, w, i, lane)) * czl.ig;
                    const T gr = (Ps(sp, w, i, lr) - Ps(sm, w, i, lr)) * czl.ig;
                    v -= T(ez) * k.hc * (fE.tl * gl + fE.tr * gr);
                }
                fEx[XS3<QQ>(i, 0)] = fma(k.a_f, v, horner3(k.hf, i, phib));
            }
        }
        // north y-face (rows 0..NW-2, lanes 1..30): shared with the row above as its south face
        if (w <= NW - 2 && interior_col) {
            const int wu = w + 1;
            const T phib = (T(1) - fN.w) * Ms(so, w, 0, lane) + fN.w * Ms(so, wu, 0, lane) +
                           fN.hcd * (Ms(so, w, 2, lane) - Ms(so, wu, 2, lane)) -
                           k.hc * (fN.tl * ((Ms(so, w, 1, l2) - Ms(so, w, 1, l1)) * cxj.ig +
                                            (Ms(sp, w, 3, lane) - Ms(sm, w, 3, lane)) * czl.ig) +
                                   fN.tr * ((Ms(so, wu, 1, l2) - Ms(so, wu, 1, l1)) * cxj.ig +
                                            (Ms(sp, wu, 3, lane) - Ms(sm, wu, 3, lane)) * czl.ig));
#pragma unroll
            for (int i = 0; i < QQ; ++i) {
                if (XS3<QQ>(i, 1) < 0) continue;
                const int en = E3<QQ>(i, 1), ex = E3<QQ>(i, 0), ez = E3<QQ>(i, 2);
                T v = ((T(1) - fN.w) + T(en) * fN.hcd) * Ps(so, w, i, lane) + (fN.w - T(en) * fN.hcd) * Ps(so, wu, i, lane);
                if (ex != 0) {
                    const T gl = (Ps(so, w, i, l2) - Ps(so, w, i, l1)) * cxj.ig;
                    const T gr = (Ps(so, wu, i, l2) - Ps(so, wu, i, l1)) * cxj.ig;
                    v -= T(ex) * k.hc * (fN.tl * gl + fN.tr * gr);
                }
                if (ez != 0) {
                    const T gl = (Ps(sp, w, i, lane) - Ps(sm, w, i, lane)) * czl.ig;
                    const T gr = (Ps(sp, wu, i, lane) - Ps(sm, wu, i, lane)) * czl.ig;
                    v -= T(ez) * k.hc * (fN.tl * gl + fN.tr * gr);
                }
                const T f = fma(k.a_f, v, horner3(k.hf, i, phib));
                fNy[XS3<QQ>(i, 1)] = f;
                sY[(w * NCROSS + XS3<QQ>(i, 1)) * 32 + lane] = f;
            }
        }
        // top z-face (interior rows)
        if (interior_row) z_face(so, sp, a.fm[2][z + 2], fTz);
        // west x-face: the east face of the lane to the left
        T fWx[NCROSS];
#pragma unroll
        for (int s = 0; s < NCROSS; ++s) fWx[s] = __shfl_up_sync(0xffffffffu, fEx[s], 1);
        __syncthreads();  // south faces in sY; every read of slot sm is done
        if (updates) {
            const long long c = ((long long)z * ny + kk) * nx + j;
#pragma unroll
            for (int i = 0; i < QQ; ++i) {
                const T P = Ps(so, w, i, lane);
                T v = fma(k.third, P - Fs(so, i), P);  // ftilde^+ (Eq. 2.23)
                if (XS3<QQ>(i, 0) >= 0)
                    v = fma(-T(E3<QQ>(i, 0)) * cxj.r, fEx[XS3<QQ>(i, 0)] - fWx[XS3<QQ>(i, 0)], v);
                if (XS3<QQ>(i, 1) >= 0)
                    v = fma(-T(E3<QQ>(i, 1)) * cyk.r, fNy[XS3<QQ>(i, 1)] - sY[((w - 1) * NCROSS + XS3<QQ>(i, 1)) * 32 + lane], v);
                if (XS3<QQ>(i, 2) >= 0)
                    v = fma(-T(E3<QQ>(i, 2)) * czl.r, fTz[XS3<QQ>(i, 2)] - fB[XS3<QQ>(i, 2)], v);
                a.fout[i * a.plane + c] = v;
            }
        }
#pragma unroll
        for (int s = 0; s < NCROSS; ++s) fB[s] = fTz[s];
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // the last prefetch lands before exit
}

// ---------------------------------------------------------------------------
// step3d_vp: the same dataflow in single precision on velocity pairs
// ---------------------------------------------------------------------------
//
// Every moving velocity is paired with its opposite (D3Q19: 9 pairs, D3Q15: 7)
// and a pair is one float2: the rings hold P and ftilde of a cell as pairs (one
// 64-bit shared-memory access per pair) and the per-velocity arithmetic runs on
// the packed FP32 instructions.  The second velocity of a pair is the opposite
// of the first, so each per-pair weight has the form (a + s b, a - s b) with s
// the direction sign of the first.  The rest velocity never crosses a face: its
// P stays in a register until the update.

using dugks::F2;
using dugks::f2;
using dugks::fma2;
using dugks::sgn2;
using dugks::shfl_up2;
using dugks::fence_mbar_init;
using dugks::fence_proxy_async_smem;
using dugks::mbar_arrive_expect_tx;
using dugks::mbar_init;
using dugks::mbar_wait_bounded;
using dugks::smem_u32;
using dugks::tma_load_4d;

// the opposite of velocity i
template <int QQ>
__host__ __device__ constexpr int OPP3(int i) {
    for (int j = 0; j < QQ; ++j)
        if (E3<QQ>(j, 0) == -E3<QQ>(i, 0) && E3<QQ>(j, 1) == -E3<QQ>(i, 1) && E3<QQ>(j, 2) == -E3<QQ>(i, 2)) return j;
    return -1;
}
// pair q = (PA3(q), PB3(q)): the pairs in order of their first velocity, the second its
// opposite (tables spelled out so that they fold to constants after unrolling)
template <int QQ>
__host__ __device__ constexpr int PA3(int q) { return QQ == 19 ? 2 * q + 1 : "\1\3\5\7\10\11\12"[q]; }
template <int QQ>
__host__ __device__ constexpr int PB3(int q) { return QQ == 19 ? 2 * q + 2 : "\2\4\6\13\14\15\16"[q]; }
template <int QQ>
__host__ __device__ constexpr bool pairs_ok() {
    for (int q = 0; q < (QQ - 1) / 2; ++q)
        if (PB3<QQ>(q) != OPP3<QQ>(PA3<QQ>(q)) || (q > 0 && PA3<QQ>(q) <= PA3<QQ>(q - 1))) return false;
    return true;
}
template <int QQ>
__host__ __device__ constexpr int QE3(int q, int a) { return E3<QQ>(PA3<QQ>(q), a); }
// position of pair q among the pairs crossing a face normal to axis a (-1: parallel)
template <int QQ>
__host__ __device__ constexpr int XP3(int q, int a) {
    if (QE3<QQ>(q, a) == 0) return -1;
    int s = 0;
    for (int m = 0; m < q; ++m) s += QE3<QQ>(m, a) != 0 ? 1 : 0;
    return s;
}
constexpr int NCP = NCROSS / 2;  // crossing pairs per face of either lattice

static_assert(pairs_ok<19>() && pairs_ok<15>() && PB3<15>(3) == 11, "velocity pairs");
static_assert(XP3<19>(8, 1) == NCP - 1 && XP3<15>(6, 2) == NCP - 1 && XP3<19>(0, 1) == -1, "crossing pairs");

template <int QQ, int NC>
struct Consts3P {
    static constexpr int NP = (QQ - 1) / 2;
    float2 hbp[NP][NC];  // per pair: b_bp (feq_A, feq_B) coefficients in powers of phi
    float2 hf[NP][NC];   // per pair: b_f (feq_A, feq_B)
    float feq[QQ][NC];   // feq_i (ghosts)
    float2 a_bp2, a_f2, third2;
    float a_bp, b_bp, third, hc;
    float bcv[6];
};

template <int QQ, int NC>
__device__ __forceinline__ F2 hbp3(const Consts3P<QQ, NC>& k, int q, F2 x) {
    F2 s{k.hbp[q][NC - 1]};
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma2(s, x, F2{k.hbp[q][m]});
    return s;
}
template <int QQ, int NC>
__device__ __forceinline__ F2 hf3(const Consts3P<QQ, NC>& k, int q, F2 x) {
    F2 s{k.hf[q][NC - 1]};
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma2(s, x, F2{k.hf[q][m]});
    return s;
}

// TMA staging of ftilde: per warp and plane one box of 36 columns x 1 row x 1 plane x QQ
// velocities ([QQ][36] floats), each box 128-byte aligned
constexpr int BOX3W = 36;
template <int QQ>
__host__ __device__ constexpr int box3_bytes() { return (QQ * BOX3W * 4 + 127) / 128 * 128; }

// shared memory of step3d_vp: P pairs, north faces and moments of three planes, then the
// ftilde ring (TM: TMA boxes and their mbarriers, with 128 bytes of alignment slack;
// else per-thread cp.async slots)
template <int QQ, int NW, bool TM>
__host__ __device__ constexpr size_t smem3_vp() {
    constexpr int NP = (QQ - 1) / 2;
    return size_t(3 * NW * NP * 32 + NW * NCP * 32) * sizeof(float2) + size_t(3 * NW * 4 * 32) * sizeof(float) +
           (TM ? size_t(3 * NW) * (box3_bytes<QQ>() + 8) + 128
               : size_t(3 * NW * NP * 32) * sizeof(float2) + size_t(3 * NW * 32) * sizeof(float));
}

// TM: ftilde arrives by TMA (tin: 4-D map of the source state, x = nx a multiple of 4);
// else by per-thread cp.async copies
template <int QQ, int NC, int NW, bool TM>
__global__ void __launch_bounds__(NW * 32, 1)
    step3d_vp(const __grid_constant__ CUtensorMap tin, const Args3<float> a, const Consts3P<QQ, NC> k) {
    constexpr int NP = (QQ - 1) / 2;
    constexpr int BOXB = box3_bytes<QQ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F2* sP = reinterpret_cast<F2*>(smem_raw);  // [3][NW][NP][32]: P pairs of three planes
    F2* sY = sP + 3 * NW * NP * 32;            // [NW][NCP][32]: north y-face f of each row
    float* sM = reinterpret_cast<float*>(sY + NW * NCP * 32);  // [3][NW][4][32]: moments M0, Mx, My, Mz
    unsigned char* ring = reinterpret_cast<unsigned char*>(sM + 3 * NW * 4 * 32);
    // !TM: [3][NW][NP][32] ftilde pairs and [3][NW][32] rest ftilde; TM: [3][NW] boxes + mbarriers
    F2* sF = reinterpret_cast<F2*>(ring);
    float* sF0 = reinterpret_cast<float*>(sF + 3 * NW * NP * 32);
    unsigned char* boxes = ring + ((128u - (smem_u32(ring) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(boxes + size_t(3 * NW) * BOXB);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x0 = blockIdx.x * 30, y0 = blockIdx.y * (NW - 2), z0 = blockIdx.z * a.zseg;
    if (z0 >= a.nz) return;  // uniform over the CTA
    const int z1 = min(z0 + a.zseg, a.nz);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int j = x0 - 1 + lane, kk = y0 - 1 + w;
    const int sj = wrapc(j, nx, a.per[0]), sk = wrapc(kk, ny, a.per[1]);
    const bool gx = !a.per[0] && (j < 0 || j >= nx), gy = !a.per[1] && (kk < 0 || kk >= ny);
    const int jm = min(max(j, -1), nx), km = min(max(kk, -1), ny);
    const FaceM<float> fE = a.fm[0][jm + 2], fN = a.fm[1][km + 2];
    const CellM<float> cxj = a.cm[0][jm + 1], cyk = a.cm[1][km + 1];
    const bool interior_row = w >= 1 && w <= NW - 2;
    const bool interior_col = lane >= 1 && lane <= 30;
    const bool updates = interior_row && interior_col && j < nx && kk < ny;
    const int l1 = max(lane - 1, 0), l2 = min(lane + 1, 31);
    const int w1 = max(w - 1, 0), w2 = min(w + 1, NW - 1);

    auto Ps = [&](int slot, int ww, int q, int l) -> F2 { return sP[((slot * NW + ww) * NP + q) * 32 + l]; };
    auto Ms = [&](int slot, int ww, int m, int l) -> float { return sM[((slot * NW + ww) * 4 + m) * 32 + l]; };
    auto slot_of = [&](int zz) { return (zz - z0 + 1) % 3; };
    // TM: this lane's column in its warp's box, or (edge strips) a periodic image or a clamped
    // ghost source read from global memory
    const int xs = (x0 - 1) & ~3;
    const int col = j - xs;
    const bool from_box = j >= 0 && j < nx;
    int issued = z0 - 2, consumed = z0 - 2;  // TM: the last plane whose box was requested / awaited
    bool fail = false;
    if (TM) {
        if (lane == 0) {
            for (int sl = 0; sl < 3; ++sl) mbar_init(&bars[sl * NW + w], 1);
            fence_mbar_init();
        }
        __syncwarp();
    }
    // start the copy of this thread's ftilde of plane zz into its slots of sF and sF0 (TM: the
    // warp's box of plane zz, requested by lane 0 once every lane has read the slot's last plane)
    auto prefetch = [&](int zz) {
        const long long c = ((long long)wrapc(zz, nz, a.per[2]) * ny + sk) * nx + sj;
        const int sl = slot_of(zz);
        if constexpr (TM) {
            __syncwarp();
            if (lane == 0) {
                uint64_t* bar = &bars[sl * NW + w];
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, uint32_t(QQ * BOX3W * 4));
                tma_load_4d(boxes + size_t(sl * NW + w) * BOXB, &tin, bar, xs, sk, wrapc(zz, nz, a.per[2]), 0);
            }
            issued = zz;
            return;
        }
        auto cp4 = [&](const void* dst, int i) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                             static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                         "l"(a.fin + i * a.plane + c));
        };
        cp4(sF0 + (sl * NW + w) * 32 + lane, 0);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            F2* d = sF + ((sl * NW + w) * NP + q) * 32 + lane;
            cp4(&d->v.x, PA3<QQ>(q));
            cp4(&d->v.y, PB3<QQ>(q));
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    // P of plane zz (already prefetched) into ring slot `slot`, its rest component returned;
    // then prefetch plane `next`
    auto compute_P = [&](int zz, int slot, int next) -> float {
        const bool gz = !a.per[2] && (zz < 0 || zz >= nz);
        F2 F[NP];
        float F0;
        if constexpr (TM) {
            // the n-th use of a slot waits for phase n & 1 of its mbarrier (bounded); after a
            // timeout no further wait is made and the copies from the failed one on are drained
            // at exit
            if (!fail) {
                if (mbar_wait_bounded(&bars[slot * NW + w], uint32_t(((zz - z0 + 1) / 3) & 1), 2000000000ull))
                    consumed = zz;
                else
                    fail = true;
            }
            if (from_box) {
                const float* bx = reinterpret_cast<const float*>(boxes + size_t(slot * NW + w) * BOXB) + col;
                F0 = bx[0];
#pragma unroll
                for (int q = 0; q < NP; ++q) F[q] = f2(bx[PA3<QQ>(q) * BOX3W], bx[PB3<QQ>(q) * BOX3W]);
            } else {
                const float* src = a.fin + ((long long)wrapc(zz, nz, a.per[2]) * ny + sk) * nx + sj;
                F0 = src[0];
#pragma unroll
                for (int q = 0; q < NP; ++q) F[q] = f2(src[PA3<QQ>(q) * a.plane], src[PB3<QQ>(q) * a.plane]);
            }
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            F0 = sF0[(slot * NW + w) * 32 + lane];
#pragma unroll
            for (int q = 0; q < NP; ++q) F[q] = sF[((slot * NW + w) * NP + q) * 32 + lane];
        }
        F2 fs = f2(0.f);
#pragma unroll
        for (int q = 0; q < NP; ++q) fs = fs + F[q];
        const float phi = F0 + (fs.v.x + fs.v.y);
        // the slots of plane next held plane next-3, whose update this thread has done
        prefetch(next);
        const F2 phi2 = f2(phi);
        F2 P[NP];
        F2 hs = f2(0.f);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const F2 h = hbp3(k, q, phi2);
            P[q] = fma2(F2{k.a_bp2}, F[q], h);
            hs = hs + h;
        }
        float P0 = fmaf(k.a_bp, F0, fmaf(k.b_bp, phi, -(hs.v.x + hs.v.y)));  // rest velocity via the zeroth moment
        if (gx || gy || gz) {  // mirrored ghost: P_g = feq(2 bv - phi) + P - feq(phi)
            const float bv = gx ? (j < 0 ? k.bcv[0] : k.bcv[1])
                                : (gy ? (kk < 0 ? k.bcv[2] : k.bcv[3]) : (zz < 0 ? k.bcv[4] : k.bcv[5]));
            const float pg = 2.f * bv - phi;
            auto dfe = [&](int i) { return horner3(k.feq, i, pg) - horner3(k.feq, i, phi); };
#pragma unroll
            for (int q = 0; q < NP; ++q) P[q] = P[q] + f2(dfe(PA3<QQ>(q)), dfe(PB3<QQ>(q)));
            P0 += dfe(0);
        }
        F2 s2 = f2(0.f);
        float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            sP[((slot * NW + w) * NP + q) * 32 + lane] = P[q];
            s2 = s2 + P[q];
            const float d = P[q].v.x - P[q].v.y;  // e_a P of the pair = e_a(A) (P_A - P_B)
            if (QE3<QQ>(q, 0) != 0) mx += QE3<QQ>(q, 0) > 0 ? d : -d;
            if (QE3<QQ>(q, 1) != 0) my += QE3<QQ>(q, 1) > 0 ? d : -d;
            if (QE3<QQ>(q, 2) != 0) mz += QE3<QQ>(q, 2) > 0 ? d : -d;
        }
        float* M = sM + (slot * NW + w) * 4 * 32 + lane;
        M[0] = P0 + (s2.v.x + s2.v.y);
        M[32] = mx;
        M[64] = my;
        M[96] = mz;
        return P0;
    };

    // tangential part of a face reconstruction: tl times the central difference of the
    // lower/left cell plus tr times that of the other cell, for one tangential axis
    auto tang = [&](const F2& lm, const F2& lp, const F2& rm, const F2& rp, float tl, float tr) {
        return fma2(f2(tl), lp - lm, f2(tr) * (rp - rm));
    };
    // f of the pairs crossing the z-face between ring slots lo (below) and hi (above)
    auto z_face = [&](int lo, int hi, const FaceM<float>& fz, F2 (&out)[NCP]) {
        const float phib = (1.f - fz.w) * Ms(lo, w, 0, lane) + fz.w * Ms(hi, w, 0, lane) +
                           fz.hcd * (Ms(lo, w, 3, lane) - Ms(hi, w, 3, lane)) -
                           k.hc * (fz.tl * ((Ms(lo, w, 1, l2) - Ms(lo, w, 1, l1)) * cxj.ig +
                                            (Ms(lo, w2, 2, lane) - Ms(lo, w1, 2, lane)) * cyk.ig) +
                                   fz.tr * ((Ms(hi, w, 1, l2) - Ms(hi, w, 1, l1)) * cxj.ig +
                                            (Ms(hi, w2, 2, lane) - Ms(hi, w1, 2, lane)) * cyk.ig));
        const F2 phib2 = f2(phib);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            if (XP3<QQ>(q, 2) < 0) continue;
            const int en = QE3<QQ>(q, 2), ex = QE3<QQ>(q, 0), ey = QE3<QQ>(q, 1);
            F2 v = fma2(sgn2(1.f - fz.w, fz.hcd, en), Ps(lo, w, q, lane), sgn2(fz.w, -fz.hcd, en) * Ps(hi, w, q, lane));
            if (ex != 0)
                v = fma2(sgn2(0.f, -k.hc * cxj.ig, ex),
                         tang(Ps(lo, w, q, l1), Ps(lo, w, q, l2), Ps(hi, w, q, l1), Ps(hi, w, q, l2), fz.tl, fz.tr), v);
            if (ey != 0)
                v = fma2(sgn2(0.f, -k.hc * cyk.ig, ey),
                         tang(Ps(lo, w1, q, lane), Ps(lo, w2, q, lane), Ps(hi, w1, q, lane), Ps(hi, w2, q, lane), fz.tl,
                              fz.tr), v);
            out[XP3<QQ>(q, 2)] = fma2(F2{k.a_f2}, v, hf3(k, q, phib2));
        }
    };

    // pipeline fill: planes z0-1 and z0, and the bottom face of plane z0
    prefetch(z0 - 1);
    compute_P(z0 - 1, 0, z0);
    float P0n = compute_P(z0, 1, z0 + 1);  // rest component of P of the plane being updated
    // TM: a bounded wait that expired anywhere in the CTA stops every warp at the same barrier
    bool stop = false;
    if constexpr (TM) stop = __syncthreads_or(fail) != 0;
    else __syncthreads();
    F2 fB[NCP];
#pragma unroll
    for (int s = 0; s < NCP; ++s) fB[s] = f2(0.f);
    if (interior_row && !stop) z_face(0, 1, a.fm[2][z0 + 1], fB);

    // z metrics of the plane being updated and of its top face, loaded a plane ahead
    CellM<float> czn = a.cm[2][z0 + 1];
    FaceM<float> fzn = a.fm[2][z0 + 2];
    for (int z = z0; z < z1 && !stop; ++z) {
        const int sm = (z - z0) % 3, so = (z - z0 + 1) % 3, sp = (z - z0 + 2) % 3;
        const float P0 = P0n;
        const CellM<float> czl = czn;
        const FaceM<float> fzt = fzn;
        czn = a.cm[2][min(z + 2, nz)];
        fzn = a.fm[2][min(z + 3, nz + 1)];
        P0n = compute_P(z + 1, sp, z + 2);
        if constexpr (TM) {
            if (__syncthreads_or(fail)) break;
        } else {
            __syncthreads();
        }
        F2 fEx[NCP], fNy[NCP], fTz[NCP];
#pragma unroll
        for (int s = 0; s < NCP; ++s) fEx[s] = fNy[s] = fTz[s] = f2(0.f);
        // east x-face (lanes 0..30 of the interior rows)
        if (interior_row && lane <= 30) {
            const int lr = lane + 1;
            const float phib = (1.f - fE.w) * Ms(so, w, 0, lane) + fE.w * Ms(so, w, 0, lr) +
                               fE.hcd * (Ms(so, w, 1, lane) - Ms(so, w, 1, lr)) -
                               k.hc * (fE.tl * ((Ms(so, w2, 2, lane) - Ms(so, w1, 2, lane)) * cyk.ig +
                                                (Ms(sp, w, 3, lane) - Ms(sm, w, 3, lane)) * czl.ig) +
                                       fE.tr * ((Ms(so, w2, 2, lr) - Ms(so, w1, 2, lr)) * cyk.ig +
                                                (Ms(sp, w, 3, lr) - Ms(sm, w, 3, lr)) * czl.ig));
            const F2 phib2 = f2(phib);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                if (XP3<QQ>(q, 0) < 0) continue;
                const int en = QE3<QQ>(q, 0), ey = QE3<QQ>(q, 1), ez = QE3<QQ>(q, 2);
                F2 v = fma2(sgn2(1.f - fE.w, fE.hcd, en), Ps(so, w, q, lane), sgn2(fE.w, -fE.hcd, en) * Ps(so, w, q, lr));
                if (ey != 0)
                    v = fma2(sgn2(0.f, -k.hc * cyk.ig, ey),
                             tang(Ps(so, w1, q, lane), Ps(so, w2, q, lane), Ps(so, w1, q, lr), Ps(so, w2, q, lr), fE.tl,
                                  fE.tr), v);
                if (ez != 0)
                    v = fma2(sgn2(0.f, -k.hc * czl.ig, ez),
                             tang(Ps(sm, w, q, lane), Ps(sp, w, q, lane), Ps(sm, w, q, lr), Ps(sp, w, q, lr), fE.tl,
                                  fE.tr), v);
                fEx[XP3<QQ>(q, 0)] = fma2(F2{k.a_f2}, v, hf3(k, q, phib2));
            }
        }
        // north y-face (rows 0..NW-2, lanes 1..30): shared with the row above as its south face
        if (w <= NW - 2 && interior_col) {
            const int wu = w + 1;
            const float phib = (1.f - fN.w) * Ms(so, w, 0, lane) + fN.w * Ms(so, wu, 0, lane) +
                               fN.hcd * (Ms(so, w, 2, lane) - Ms(so, wu, 2, lane)) -
                               k.hc * (fN.tl * ((Ms(so, w, 1, l2) - Ms(so, w, 1, l1)) * cxj.ig +
                                                (Ms(sp, w, 3, lane) - Ms(sm, w, 3, lane)) * czl.ig) +
                                       fN.tr * ((Ms(so, wu, 1, l2) - Ms(so, wu, 1, l1)) * cxj.ig +
                                                (Ms(sp, wu, 3, lane) - Ms(sm, wu, 3, lane)) * czl.ig));
            const F2 phib2 = f2(phib);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                if (XP3<QQ>(q, 1) < 0) continue;
                const int en = QE3<QQ>(q, 1), ex = QE3<QQ>(q, 0), ez = QE3<QQ>(q, 2);
                F2 v = fma2(sgn2(1.f - fN.w, fN.hcd, en), Ps(so, w, q, lane), sgn2(fN.w, -fN.hcd, en) * Ps(so, wu, q, lane));
                if (ex != 0)
                    v = fma2(sgn2(0.f, -k.hc * cxj.ig, ex),
                             tang(Ps(so, w, q, l1), Ps(so, w, q, l2), Ps(so, wu, q, l1), Ps(so, wu, q, l2), fN.tl,
                                  fN.tr), v);
                if (ez != 0)
                    v = fma2(sgn2(0.f, -k.hc * czl.ig, ez),
                             tang(Ps(sm, w, q, lane), Ps(sp, w, q, lane), Ps(sm, wu, q, lane), Ps(sp, wu, q, lane), fN.tl,
                                  fN.tr), v);
                const F2 f = fma2(F2{k.a_f2}, v, hf3(k, q, phib2));
                fNy[XP3<QQ>(q, 1)] = f;
                sY[(w * NCP + XP3<QQ>(q, 1)) * 32 + lane] = f;
            }
        }
        // top z-face (interior rows)
        if (interior_row) z_face(so, sp, fzt, fTz);
        // west x-face: the east face of the lane to the left
        F2 fWx[NCP];
#pragma unroll
        for (int s = 0; s < NCP; ++s) fWx[s] = shfl_up2(fEx[s]);
        // Row w's update needs the south face of row w - 1 (sY), and the next compute_P of
        // row w overwrites, in slot sm, data that row w - 1 has read for its faces: so each
        // row waits for the row below only (named barrier w: row w - 1 arrives, row w waits)
        // instead of for the whole CTA.  Every barrier id 1 .. NW-1 has exactly one arriving
        // and one waiting warp per plane.
        if (w <= NW - 2) asm volatile("bar.arrive %0, 64;" ::"r"(w + 1) : "memory");
        if (w >= 1) asm volatile("bar.sync %0, 64;" ::"r"(w) : "memory");
        if (updates) {  // (an updating lane's column is always in its warp's box)
            const long long c = ((long long)z * ny + kk) * nx + j;
            const float* bx = reinterpret_cast<const float*>(boxes + size_t(so * NW + w) * BOXB) + col;
            auto Fso = [&](int q) -> F2 {
                if constexpr (TM) return f2(bx[PA3<QQ>(q) * BOX3W], bx[PB3<QQ>(q) * BOX3W]);
                else return sF[((so * NW + w) * NP + q) * 32 + lane];
            };
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const F2 P = Ps(so, w, q, lane);
                F2 v = fma2(F2{k.third2}, P - Fso(q), P);  // ftilde^+ (Eq. 2.23)
                if (XP3<QQ>(q, 0) >= 0)
                    v = fma2(sgn2(0.f, -cxj.r, QE3<QQ>(q, 0)), fEx[XP3<QQ>(q, 0)] - fWx[XP3<QQ>(q, 0)], v);
                if (XP3<QQ>(q, 1) >= 0)
                    v = fma2(sgn2(0.f, -cyk.r, QE3<QQ>(q, 1)),
                             fNy[XP3<QQ>(q, 1)] - sY[((w - 1) * NCP + XP3<QQ>(q, 1)) * 32 + lane], v);
                if (XP3<QQ>(q, 2) >= 0)
                    v = fma2(sgn2(0.f, -czl.r, QE3<QQ>(q, 2)), fTz[XP3<QQ>(q, 2)] - fB[XP3<QQ>(q, 2)], v);
                if constexpr (TM) {  // 32-bit plane offsets: the host takes TM below 2^32 elements
                    float* o = a.fout + c;
                    const uint32_t pl = uint32_t(a.plane);
                    o[uint32_t(PA3<QQ>(q)) * pl] = v.v.x;
                    o[uint32_t(PB3<QQ>(q)) * pl] = v.v.y;
                } else {
                    a.fout[PA3<QQ>(q) * a.plane + c] = v.v.x;
                    a.fout[PB3<QQ>(q) * a.plane + c] = v.v.y;
                }
            }
            a.fout[c] = fmaf(k.third, P0 - (TM ? bx[0] : sF0[(so * NW + w) * 32 + lane]), P0);
        }
#pragma unroll
        for (int s = 0; s < NCP; ++s) fB[s] = fTz[s];
    }
    if constexpr (TM) {
        // the boxes still in flight land before the CTA exits (bounded waits)
        if (fail) atomicOr(a.err, 1);
        for (int zz = consumed + 1; zz <= issued; ++zz)
            mbar_wait_bounded(&bars[slot_of(zz) * NW + w], uint32_t(((zz - z0 + 1) / 3) & 1), 100000000ull);
    } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");  // the last prefetch lands before exit
    }
}

// phi = sum_i ftilde_i (optional output) and per-block partial sums of |V| phi in double
template <typename T, int QQ>
__global__ void __launch_bounds__(256) phi_mass3(const T* __restrict__ f, T* __restrict__ phi, int nx, int ny, int nz,
                                                 const double* __restrict__ dxv, const double* __restrict__ dyv,
                                                 const double* __restrict__ dzv, double* __restrict__ partial) {
    const long long n = (long long)nx * ny * nz;
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int j = int(c % nx);
        const long long r = c / nx;
        const int kk = int(r % ny), l = int(r / ny);
        T s = T(0);
#pragma unroll
        for (int i = 0; i < QQ; ++i) s += f[i * n + c];
        if (phi) phi[c] = s;
        acc += dxv[j] * dyv[kk] * dzv[l] * double(s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < int(blockDim.x >> 5); ++q) s += ws[q];
        partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) sum3(const double* __restrict__ partial, int n, double* __restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < int(blockDim.x >> 5); ++q) s += ws[q];
        *out = s;
    }
}

// ftilde = feq(phi0) (opening of Section 4); phi0 [nz][ny][nx]
template <typename T, int QQ, int NC, typename Tin>
__global__ void init3(const Tin* __restrict__ phi0, T* __restrict__ f, long long n, const Consts3<T, QQ, NC> k) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const T p = T(phi0[c]);
#pragma unroll
        for (int i = 0; i < QQ; ++i) f[i * n + c] = horner3(k.feq, i, p);
    }
}

}  // namespace dugks3

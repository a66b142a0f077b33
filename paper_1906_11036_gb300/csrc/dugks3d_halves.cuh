// dugks3d_halves.cuh -- the 3-D DUGKS step (arXiv:1906.11036, Section 2 with the
// D3Q15 / D3Q19 sets of Eqs. 2.28 / 2.6) in single precision with every face built
// from two halves, one per cell.
//
// A face value fbar_i (Eqs. 2.19, 2.20, 2.26) is linear in the two cells' P = fbar^+
// and in their slopes along the axes tangential to the face:
//   fbar_i = w_L(i) P_i(L) + w_R(i) P_i(R) - h c sum_t e_t,i [tl s_t P_i(L) + tr s_t P_i(R)]
// so it splits into a half that only needs cell L and a half that only needs cell R.
// Each cell forms its slopes s_t P_i once (central differences, as the scalar kernel)
// and from them both halves of each of its faces; phi_b = sum_i fbar_i splits the same
// way in the moments M0 = phi, M_a = sum_i e_a,i P_i and the tangential slopes s_t M_t.
//
// A CTA of NW warps owns 30 columns (lanes 1..30; lanes 0 and 31 are the x-halo) by
// NW - 2 rows (warps 1..NW-2; warps 0 and NW-1 are the y-halo) and marches up a segment
// of z-planes.  Pass pp (planes z0-1 .. z1) forms P of plane pp and updates plane
// z = pp - 1:
//   1. P, phi and the moments of plane pp from its ftilde box (Eq. 2.21), the z-slopes
//      of plane z, and the two y-face halves of plane z;
//   2. into shared memory: P of plane pp for the pairs that have tangential slopes
//      (and Mx, My), and the y-face halves of plane z;  one CTA barrier;
//   3. x-faces of plane z: own half plus the right neighbour's by shuffle; y-faces:
//      own half plus the neighbour row's from shared memory; ftilde^+ (Eq. 2.23) plus
//      the x and y fluxes (Eq. 2.12);
//   4. x- and y-slopes of plane pp from shared memory, its two z-face halves; the
//      z-face between z and pp completes (the lower half was formed one pass earlier);
//   5. the z fluxes complete the update of plane z, which is written.
// The shared buffers of steps 2 alternate between passes, so one barrier per plane
// separates every write from the reads of the pass before.
//
// ftilde of each warp's row arrives by one 4-D TMA box (36 columns x 1 x 1 x Q) per
// plane into a three-plane ring per warp (planes z, pp, pp+1), with bounded mbarrier
// waits; a timeout anywhere stops the whole CTA at its next barrier and is reported in
// the error word.
//
// Every per-pair quantity (pair directions, crossing and slope indices) is a compile-time
// constant of the code that uses it (sfor below): evaluated at run time, the velocity
// tables cost more than the arithmetic.  The library runs this kernel for D3Q15 (256^3:
// 1166 us per step against 1214 for the face kernel of dugks3d_kernels.cuh); for D3Q19 the
// face kernel is faster (1144 us against 1188-1211), with the live state here at 158-164
// registers.
#pragma once
#include <type_traits>
#include <utility>

#include "dugks3d_kernels.cuh"

namespace dugks3 {

// f(std::integral_constant<int, q>) for q = 0 .. N-1: the per-pair code sees q, and every
// table entry derived from it, as a compile-time constant (if constexpr drops what a pair
// does not need)
template <typename F, int... I>
__device__ __forceinline__ void sfor_(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
    sfor_(f, std::make_integer_sequence<int, N>{});
}

// number of nonzero direction components of pair q
template <int QQ>
__host__ __device__ constexpr int NZ3(int q) {
    return (QE3<QQ>(q, 0) != 0 ? 1 : 0) + (QE3<QQ>(q, 1) != 0 ? 1 : 0) + (QE3<QQ>(q, 2) != 0 ? 1 : 0);
}
// pair q needs its slope along axis t: it moves along t and crosses faces of another axis
template <int QQ>
__host__ __device__ constexpr bool SL3(int q, int t) {
    return QE3<QQ>(q, t) != 0 && NZ3<QQ>(q) >= 2;
}
// position of pair q among the pairs with tangential slopes (-1: none)
template <int QQ>
__host__ __device__ constexpr int SP3(int q) {
    if (NZ3<QQ>(q) < 2) return -1;
    int s = 0;
    for (int m = 0; m < q; ++m) s += NZ3<QQ>(m) >= 2 ? 1 : 0;
    return s;
}
template <int QQ>
__host__ __device__ constexpr int NSP3() {
    int s = 0;
    for (int q = 0; q < (QQ - 1) / 2; ++q) s += NZ3<QQ>(q) >= 2 ? 1 : 0;
    return s;
}
static_assert(NSP3<19>() == 6 && NSP3<15>() == 4 && SP3<19>(8) == 5 && SP3<19>(2) == -1, "slope pairs");

// shared memory of step3d_hv: two alternating sets of (slope-pair P, Mx, My, Mz, y-face
// halves and their phi_b parts), the column and row metric tables, then the TMA ring with its mbarriers (128 bytes of
// alignment slack)
template <int QQ, int NW>
__host__ __device__ constexpr size_t smem3_hv() {
    return size_t(2 * NW * NSP3<QQ>() * 32 + 2 * NW * 2 * NCP * 32) * sizeof(float2) +
           size_t(2 * NW * 3 * 32 + 2 * NW * 2 * 32 + 10 * 32 + NW * 10) * sizeof(float) +
           size_t(3 * NW) * (box3_bytes<QQ>() + 8) + 128;
}

#ifndef DUGKS_3D_HV_NW
#define DUGKS_3D_HV_NW 12
#endif

template <int QQ, int NC, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
    step3d_hv(const __grid_constant__ CUtensorMap tin, const Args3<float> a, const Consts3P<QQ, NC> k) {
    constexpr int NP = (QQ - 1) / 2;
    constexpr int NS = NSP3<QQ>();
    constexpr int BOXB = box3_bytes<QQ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F2* sS = reinterpret_cast<F2*>(smem_raw);                           // [2][NW][NS][32] P of the slope pairs
    F2* sH = sS + 2 * NW * NS * 32;                                     // [2][NW][2][NCP][32] y-face halves
    float* sSM = reinterpret_cast<float*>(sH + 2 * NW * 2 * NCP * 32);  // [2][NW][3][32] Mx, My, Mz
    float* sHP = sSM + 2 * NW * 3 * 32;                                 // [2][NW][2][32] phi_b halves (y)
    float* sXm = sHP + 2 * NW * 2 * 32;  // [10][32] east face, west face, cell metrics of each lane's column
    float* sYm = sXm + 10 * 32;          // [NW][10] north face, south face, cell metrics of each warp's row
    unsigned char* ring = reinterpret_cast<unsigned char*>(sYm + NW * 10);
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
    const bool updates = w >= 1 && w <= NW - 2 && lane >= 1 && lane <= 30 && j < nx && kk < ny;
    const int l1 = max(lane - 1, 0), l2 = min(lane + 1, 31);
    const int w1 = max(w - 1, 0), w2 = min(w + 1, NW - 1);
    const int xs = (x0 - 1) & ~3;  // box origin: x * 4 bytes a multiple of 16
    const int col = j - xs;
    const bool from_box = j >= 0 && j < nx;
    const float hc = k.hc;
    // the per-column and per-row metrics live in two small shared tables (reloaded where they
    // are used, which keeps them out of the register budget)
    if (w == 0) {
        const FaceM<float> e = a.fm[0][jm + 2], o = a.fm[0][jm + 1];
        const CellM<float> c = a.cm[0][jm + 1];
        const float v[10] = {e.w, e.hcd, e.tl, e.tr, o.w, o.hcd, o.tl, o.tr, c.ig, c.r};
#pragma unroll
        for (int i = 0; i < 10; ++i) sXm[i * 32 + lane] = v[i];
    }
    if (lane == 0) {
        const FaceM<float> n = a.fm[1][km + 2], o = a.fm[1][km + 1];
        const CellM<float> c = a.cm[1][km + 1];
        const float v[10] = {n.w, n.hcd, n.tl, n.tr, o.w, o.hcd, o.tl, o.tr, c.ig, c.r};
#pragma unroll
        for (int i = 0; i < 10; ++i) sYm[w * 10 + i] = v[i];
    }
    __syncthreads();
    auto xface = [&](int o) {
        const float* p = sXm + o * 32 + lane;
        return FaceM<float>{p[0], p[32], p[64], p[96]};
    };
    auto yface = [&](int o) {
        const float* p = sYm + w * 10 + o;
        return FaceM<float>{p[0], p[1], p[2], p[3]};
    };
    auto xcell = [&]() { return CellM<float>{sXm[8 * 32 + lane], sXm[9 * 32 + lane]}; };
    auto ycell = [&]() { return CellM<float>{sYm[w * 10 + 8], sYm[w * 10 + 9]}; };

    auto slot_of = [&](int zz) { return (zz - z0 + 1) % 3; };
    auto parity_of = [&](int zz) { return uint32_t(((zz - z0 + 1) / 3) & 1); };
    auto box_of = [&](int zz) -> const float* {
        return reinterpret_cast<const float*>(boxes + size_t(slot_of(zz) * NW + w) * BOXB) + col;
    };
    int issued = z0 - 2, consumed = z0 - 2;  // the last plane whose box was requested / awaited
    bool fail = false;
    // the warp's box of plane zz, requested by lane 0 once every lane has read the slot
    auto request = [&](int zz) {
        __syncwarp();
        if (lane == 0) {
            uint64_t* bar = &bars[slot_of(zz) * NW + w];
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, uint32_t(QQ * BOX3W * 4));
            tma_load_4d(boxes + size_t(slot_of(zz) * NW + w) * BOXB, &tin, bar, xs, sk, wrapc(zz, nz, a.per[2]), 0);
        }
        issued = zz;
    };
    if (lane == 0) {
        for (int sl = 0; sl < 3; ++sl) mbar_init(&bars[sl * NW + w], 1);
        fence_mbar_init();
    }
    for (int zz = z0 - 1; zz <= z0 + 1; ++zz) request(zz);  // z1 >= z0 + 1



    // The two shared sets alternate: pass pp writes set cur = (pp - z0 + 1) & 1 (its rows of
    // slope-pair P and Mx, My, Mz of plane pp, and the y-face halves of plane z) before its
    // barrier.  Set prv then holds plane z; the neighbour rows of it are rewritten only after
    // the next barrier, so they may be read before this one.  A warp's own row is written by
    // that warp alone, so it reads its own row in program order at any time.
    auto sP = [&](int set, int ww, int sp, int l) -> F2 { return sS[((set * NW + ww) * NS + sp) * 32 + l]; };
    auto sM = [&](int set, int ww, int m, int l) -> float { return sSM[((set * NW + ww) * 3 + m) * 32 + l]; };

    // carried from pass to pass (at the start of pass pp: plane z = pp - 1): P of the pairs
    // without tangential slopes (the slope pairs are re-read from the warp's own row), the
    // rest P, phi, Mx, My, the lower half of the z-face above z and f of the z-face below z
    F2 Pz[NP], HzL[NCP], fB[NCP];
    sfor<NP>([&](auto qc) { Pz[decltype(qc)::value] = f2(0.f); });
    sfor<NCP>([&](auto sc) {
        constexpr int s_ = decltype(sc)::value;
        HzL[s_] = fB[s_] = f2(0.f);
    });
    float P0z = 0.f, phz = 0.f, mxz = 0.f, myz = 0.f, pzL = 0.f;

    for (int pp = z0 - 1; pp <= z1; ++pp) {
        const int cur = (pp - z0 + 1) & 1, prv = cur ^ 1;
        const bool upd = pp > z0;  // plane z = pp - 1 is updated in this pass
        const int z = pp - 1;
        const CellM<float> czl = a.cm[2][max(pp, 0)];                    // plane z (entry z + 1)
        const FaceM<float> fzlo = a.fm[2][pp + 1], fzhi = a.fm[2][pp + 2];  // faces below / above pp

        // 1. P of plane pp (Eq. 2.21, the rest velocity by the zeroth moment), its moments;
        //    a mirrored ghost: P_g = feq(2 bv - phi) + P - feq(phi)
        F2 Pp[NP];
        float P0p, php, mxp = 0.f, myp = 0.f, mzp = 0.f;
        {
            if (!fail) {
                if (mbar_wait_bounded(&bars[slot_of(pp) * NW + w], parity_of(pp), 2000000000ull))
                    consumed = pp;
                else
                    fail = true;
            }
            F2 F[NP];
            float F0;
            if (from_box) {
                const float* bx = box_of(pp);
                F0 = bx[0];
                sfor<NP>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    F[q] = f2(bx[PA3<QQ>(q) * BOX3W], bx[PB3<QQ>(q) * BOX3W]);
                });
            } else {
                const float* src = a.fin + ((long long)wrapc(pp, nz, a.per[2]) * ny + sk) * nx + sj;
                F0 = src[0];
                sfor<NP>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    F[q] = f2(src[PA3<QQ>(q) * a.plane], src[PB3<QQ>(q) * a.plane]);
                });
            }
            F2 fs = f2(0.f);
            sfor<NP>([&](auto qc) { fs = fs + F[decltype(qc)::value]; });
            php = F0 + (fs.v.x + fs.v.y);
            const F2 phi2 = f2(php);
            F2 hs = f2(0.f);
            sfor<NP>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                const F2 h = hbp3(k, q, phi2);
                Pp[q] = fma2(F2{k.a_bp2}, F[q], h);
                hs = hs + h;
            });
            P0p = fmaf(k.a_bp, F0, fmaf(k.b_bp, php, -(hs.v.x + hs.v.y)));
            const bool gz = !a.per[2] && (pp < 0 || pp >= nz);
            if (gx || gy || gz) {
                const float bv = gx ? (j < 0 ? k.bcv[0] : k.bcv[1])
                                    : (gy ? (kk < 0 ? k.bcv[2] : k.bcv[3]) : (pp < 0 ? k.bcv[4] : k.bcv[5]));
                const float pg = 2.f * bv - php;
                auto dfe = [&](int i) { return horner3(k.feq, i, pg) - horner3(k.feq, i, php); };
                sfor<NP>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    Pp[q] = Pp[q] + f2(dfe(PA3<QQ>(q)), dfe(PB3<QQ>(q)));
                });
                P0p += dfe(0);
                php = pg;
            }
            sfor<NP>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                const float d = Pp[q].v.x - Pp[q].v.y;  // e_a P of the pair = e_a(first) (P_A - P_B)
                if constexpr (QE3<QQ>(q, 0) != 0) mxp += QE3<QQ>(q, 0) > 0 ? d : -d;
                if constexpr (QE3<QQ>(q, 1) != 0) myp += QE3<QQ>(q, 1) > 0 ? d : -d;
                if constexpr (QE3<QQ>(q, 2) != 0) mzp += QE3<QQ>(q, 2) > 0 ? d : -d;
            });
        }

        // 2. z-slopes of plane z: P and Mz of plane z - 1 from the warp's own row of set cur
        //    (written two passes ago), read before pass pp overwrites it
        F2 Sz[NP];
        float sMz = 0.f;
        if (upd) {
            const F2 igz = f2(czl.ig);
            sfor<NP>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                if constexpr (SL3<QQ>(q, 2)) Sz[q] = (Pp[q] - sP(cur, w, SP3<QQ>(q), lane)) * igz;
            });
            sMz = (mzp - sM(cur, w, 2, lane)) * czl.ig;
        }
        // 3. P of plane pp (slope pairs) and its moments for the neighbours
        sfor<NP>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            if constexpr (SP3<QQ>(q) >= 0) sS[((cur * NW + w) * NS + SP3<QQ>(q)) * 32 + lane] = Pp[q];
        });
        sSM[((cur * NW + w) * 3 + 0) * 32 + lane] = mxp;
        sSM[((cur * NW + w) * 3 + 1) * 32 + lane] = myp;
        sSM[((cur * NW + w) * 3 + 2) * 32 + lane] = mzp;

        // 4. plane z (set prv): its y-face halves (published), its x-faces (own half plus the
        //    right neighbour's by shuffle), and ftilde^+ (Eq. 2.23) with the x fluxes
        F2 U[NP];
        float U0 = 0.f;
        if (upd) {
            sfor<NP>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                if constexpr (SP3<QQ>(q) >= 0) Pz[q] = sP(prv, w, SP3<QQ>(q), lane);
            });
            {
                const FaceM<float> fN = yface(0), fS = yface(4);
                const CellM<float> cxj = xcell();
                const F2 igx = f2(cxj.ig);
                F2 Sx[NP];
                sfor<NP>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    if constexpr (SL3<QQ>(q, 0))
                        Sx[q] = (sP(prv, w, SP3<QQ>(q), l2) - sP(prv, w, SP3<QQ>(q), l1)) * igx;
                });
                const float sMx = (sM(prv, w, 0, l2) - sM(prv, w, 0, l1)) * cxj.ig;
                sfor<NP>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    if constexpr (QE3<QQ>(q, 1) != 0) {
                        constexpr int s_ = XP3<QQ>(q, 1), ey = QE3<QQ>(q, 1);
                        F2 l = sgn2(1.f - fN.w, fN.hcd, ey) * Pz[q];
                        F2 r = sgn2(fS.w, -fS.hcd, ey) * Pz[q];
                        if constexpr (SL3<QQ>(q, 0)) {
                            l = fma2(sgn2(0.f, -hc * fN.tl, QE3<QQ>(q, 0)), Sx[q], l);
                            r = fma2(sgn2(0.f, -hc * fS.tr, QE3<QQ>(q, 0)), Sx[q], r);
                        }
                        if constexpr (SL3<QQ>(q, 2)) {
                            l = fma2(sgn2(0.f, -hc * fN.tl, QE3<QQ>(q, 2)), Sz[q], l);
                            r = fma2(sgn2(0.f, -hc * fS.tr, QE3<QQ>(q, 2)), Sz[q], r);
                        }
                        sH[(((cur * NW + w) * 2 + 0) * NCP + s_) * 32 + lane] = l;  // lower half of the north face
                        sH[(((cur * NW + w) * 2 + 1) * NCP + s_) * 32 + lane] = r;  // upper half of the south face
                    }
                });
                const float ty = sMx + sMz;
                sHP[((cur * NW + w) * 2 + 0) * 32 + lane] = fmaf(1.f - fN.w, phz, fmaf(fN.hcd, myz, -hc * fN.tl * ty));
                sHP[((cur * NW + w) * 2 + 1) * 32 + lane] = fmaf(fS.w, phz, fmaf(-fS.hcd, myz, -hc * fS.tr * ty));
            }
            F2 fEx[NCP];
            {
                const FaceM<float> fE = xface(0), fW = xface(4);
                const CellM<float> cyk = ycell();
                const F2 igy = f2(cyk.ig);
                F2 Sy[NP];
                sfor<NP>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    if constexpr (SL3<QQ>(q, 1))
                        Sy[q] = (sP(prv, w2, SP3<QQ>(q), lane) - sP(prv, w1, SP3<QQ>(q), lane)) * igy;
                });
                const float sMy = (sM(prv, w2, 1, lane) - sM(prv, w1, 1, lane)) * cyk.ig;
                const float tx = sMy + sMz;
                const float pxL = fmaf(1.f - fE.w, phz, fmaf(fE.hcd, mxz, -hc * fE.tl * tx));
                const float pxR = fmaf(fW.w, phz, fmaf(-fW.hcd, mxz, -hc * fW.tr * tx));
                const F2 pb = f2(pxL + __shfl_down_sync(0xffffffffu, pxR, 1));
                sfor<NP>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    if constexpr (QE3<QQ>(q, 0) != 0) {
                        constexpr int s_ = XP3<QQ>(q, 0), ex = QE3<QQ>(q, 0);
                        F2 l = sgn2(1.f - fE.w, fE.hcd, ex) * Pz[q];
                        F2 r = sgn2(fW.w, -fW.hcd, ex) * Pz[q];
                        if constexpr (SL3<QQ>(q, 1)) {
                            l = fma2(sgn2(0.f, -hc * fE.tl, QE3<QQ>(q, 1)), Sy[q], l);
                            r = fma2(sgn2(0.f, -hc * fW.tr, QE3<QQ>(q, 1)), Sy[q], r);
                        }
                        if constexpr (SL3<QQ>(q, 2)) {
                            l = fma2(sgn2(0.f, -hc * fE.tl, QE3<QQ>(q, 2)), Sz[q], l);
                            r = fma2(sgn2(0.f, -hc * fW.tr, QE3<QQ>(q, 2)), Sz[q], r);
                        }
                        fEx[s_] = fma2(F2{k.a_f2}, l + shfl_dn2(r), hf3(k, q, pb));  // the east face
                    }
                });
            }
            // an updating lane's column is in its box
            const float* bz = box_of(z);
            const float rx = sXm[9 * 32 + lane];
            U0 = fmaf(k.third, P0z - bz[0], P0z);
            sfor<NP>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                F2 u = fma2(F2{k.third2}, Pz[q] - f2(bz[PA3<QQ>(q) * BOX3W], bz[PB3<QQ>(q) * BOX3W]), Pz[q]);
                if constexpr (QE3<QQ>(q, 0) != 0) {  // the west face is the left neighbour's east face
                    const F2 e = fEx[XP3<QQ>(q, 0)];
                    u = fma2(sgn2(0.f, -rx, QE3<QQ>(q, 0)), e - shfl_up2(e), u);
                }
                U[q] = u;
            });
        }
        // a bounded wait that expired anywhere in the CTA stops every warp here
        if (__syncthreads_or(fail)) break;

        // 5. y-faces of plane z: the halves of this row and of the rows above and below
        if (upd) {
            auto hp = [&](int ww, int side) { return sHP[((cur * NW + ww) * 2 + side) * 32 + lane]; };
            auto hh = [&](int ww, int side, int s_) { return sH[(((cur * NW + ww) * 2 + side) * NCP + s_) * 32 + lane]; };
            const F2 pbN = f2(hp(w, 0) + hp(w2, 1)), pbS = f2(hp(w1, 0) + hp(w, 1));
            const float ry = sYm[w * 10 + 9];
            sfor<NP>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                if constexpr (QE3<QQ>(q, 1) != 0) {
                    constexpr int s_ = XP3<QQ>(q, 1);
                    const F2 fN_ = fma2(F2{k.a_f2}, hh(w, 0, s_) + hh(w2, 1, s_), hf3(k, q, pbN));
                    const F2 fS_ = fma2(F2{k.a_f2}, hh(w1, 0, s_) + hh(w, 1, s_), hf3(k, q, pbS));
                    U[q] = fma2(sgn2(0.f, -ry, QE3<QQ>(q, 1)), fN_ - fS_, U[q]);
                }
            });
        }

        // 6. x- and y-slopes of plane pp (set cur), its two z-face halves; the face between z
        //    and pp completes with the lower half formed in the previous pass
        F2 fT[NCP];
        {
            const float gxi = sXm[8 * 32 + lane], gyi = sYm[w * 10 + 8];
            const F2 igx = f2(gxi), igy = f2(gyi);
            const float sMx = (sM(cur, w, 0, l2) - sM(cur, w, 0, l1)) * gxi;
            const float sMy = (sM(cur, w2, 1, lane) - sM(cur, w1, 1, lane)) * gyi;
            const float t = sMx + sMy;
            const float pzR = fmaf(fzlo.w, php, fmaf(-fzlo.hcd, mzp, -hc * fzlo.tr * t));
            const float pzLn = fmaf(1.f - fzhi.w, php, fmaf(fzhi.hcd, mzp, -hc * fzhi.tl * t));
            const F2 pb = f2(pzL + pzR);
            sfor<NP>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                if constexpr (QE3<QQ>(q, 2) != 0) {
                    constexpr int s_ = XP3<QQ>(q, 2), ez = QE3<QQ>(q, 2), sp = SP3<QQ>(q);
                    F2 P;
                    if constexpr (sp >= 0)
                        P = sP(cur, w, sp, lane);
                    else
                        P = Pp[q];
                    F2 r = sgn2(fzlo.w, -fzlo.hcd, ez) * P;
                    F2 l = sgn2(1.f - fzhi.w, fzhi.hcd, ez) * P;
                    if constexpr (SL3<QQ>(q, 0)) {
                        const F2 g = (sP(cur, w, sp, l2) - sP(cur, w, sp, l1)) * igx;
                        r = fma2(sgn2(0.f, -hc * fzlo.tr, QE3<QQ>(q, 0)), g, r);
                        l = fma2(sgn2(0.f, -hc * fzhi.tl, QE3<QQ>(q, 0)), g, l);
                    }
                    if constexpr (SL3<QQ>(q, 1)) {
                        const F2 g = (sP(cur, w2, sp, lane) - sP(cur, w1, sp, lane)) * igy;
                        r = fma2(sgn2(0.f, -hc * fzlo.tr, QE3<QQ>(q, 1)), g, r);
                        l = fma2(sgn2(0.f, -hc * fzhi.tl, QE3<QQ>(q, 1)), g, l);
                    }
                    fT[s_] = fma2(F2{k.a_f2}, HzL[s_] + r, hf3(k, q, pb));
                    HzL[s_] = l;
                }
            });
            pzL = pzLn;
        }

        // 7. the z fluxes complete the update of plane z (Eq. 2.12)
        if (upd && updates) {
            // velocity planes by 32-bit offsets: the host runs this kernel only where the Q planes
            // hold fewer than 2^32 elements (D3Q15 256^3: 1166 us against 1186 with 64-bit ones)
            float* o = a.fout + (((long long)z * ny + kk) * nx + j);
            const uint32_t pl = uint32_t(a.plane);
            sfor<NP>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                F2 u = U[q];
                if constexpr (QE3<QQ>(q, 2) != 0)
                    u = fma2(sgn2(0.f, -czl.r, QE3<QQ>(q, 2)), fT[XP3<QQ>(q, 2)] - fB[XP3<QQ>(q, 2)], u);
                o[uint32_t(PA3<QQ>(q)) * pl] = u.v.x;
                o[uint32_t(PB3<QQ>(q)) * pl] = u.v.y;
            });
            o[0] = U0;
        }

        // plane pp becomes plane z of the next pass (its slope pairs stay in set cur)
        sfor<NP>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            if constexpr (SP3<QQ>(q) < 0) Pz[q] = Pp[q];
        });
        P0z = P0p;
        phz = php;
        mxz = mxp;
        myz = myp;
        sfor<NCP>([&](auto sc) {
            constexpr int s_ = decltype(sc)::value;
            fB[s_] = fT[s_];
        });
        // the slot of plane pp - 1 is free once its update has read it
        if (pp >= z0 && pp + 2 <= z1) request(pp + 2);
    }
    // the boxes still in flight land before the CTA exits (bounded waits)
    if (fail) atomicOr(a.err, 1);
    for (int zz = consumed + 1; zz <= issued; ++zz)
        mbar_wait_bounded(&bars[slot_of(zz) * NW + w], parity_of(zz), 100000000ull);
}

}  // namespace dugks3

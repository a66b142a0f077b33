// dugks_adjoint_rows.cuh -- the adjoint of one FP32 DUGKS step (reverse mode
// of the step of Section 2, arXiv:1906.11036) as a row march on velocity
// pairs, for grids that are periodic on both axes.
//
// The arithmetic is that of adj_tile_kernel (same face adjoints, same
// transposed weights), reorganised like the forward step: one warp owns a
// strip of 28 columns (lanes 2..29; lanes 0, 1, 30, 31 are halo columns, two
// on each side because a y-face adjoint needs the x-slope of its cell) and
// marches up a row segment.  Rows of ftilde^n and mu arrive by TMA into a
// private ring of stages.  Every face scatters its contributions to the
// adjoint of P as soon as it is formed, into three rolling accumulators for
// the rows n-2, n-1, n.  When the new row n has been processed, row n-2 has
// received every contribution (x-faces of rows n-3..n-1, y-faces below and
// above it) and is finished (Eqs. 2.21, 2.13 transposed), and its stage is
// refilled.
//
// The eight moving velocities are packed as the opposite pairs (1,3), (2,4),
// (5,7), (6,8) on the packed FP32 instructions; the second velocity of a pair
// has the opposite direction, so a per-velocity weight is a pair (a + s b,
// a - s b) with s the direction sign of the first.  Work per face:
//   * phi_b from the moments phi, Mx, My of P of the two cells (the
//     reconstruction is linear in P), so fbar is formed only for the
//     velocities that cross the face;
//   * an x-face is the sum of a half from its left cell and a half from its
//     right cell, each formed by the lane that owns the cell (one shuffle per
//     crossing value); the flux adjoint of the face returns to the right lane
//     by one shuffle per crossing value, and each lane applies its own weights;
//   * a y-face's transposed x-slope weights differ between its two rows only
//     by the face's (tl, tr), so they cross lanes once.
#pragma once
#include "dugks_adjoint.cuh"

namespace dugks {

#ifndef DUGKS_ADJ_ROWS_MIN_WARPS
#define DUGKS_ADJ_ROWS_MIN_WARPS 16
#endif
#ifndef DUGKS_ADJ_ROWS_WALL_MIN_WARPS
#define DUGKS_ADJ_ROWS_WALL_MIN_WARPS 12  // the ghost folds need more registers than 16 warps leave
#endif

struct AdjRowLayout {
    static constexpr int WI = 28;                       // owned columns per warp
    static constexpr int BOXW = 36;                     // 32 columns from (xw - 2) rounded down to 16 bytes
    static constexpr int BOX_BYTES = Q * BOXW * 4;      // one row of ftilde or mu
    static constexpr int MU_OFF = ((BOX_BYTES + 127) / 128) * 128;
    static constexpr int STAGE_BYTES = 2 * MU_OFF;      // ftilde row, then mu row
    static size_t bytes(int stages) { return size_t(stages) * (STAGE_BYTES + 8) + 128; }
};

// Constants of the FP32 adjoint on velocity pairs (pair q = (PA(q), PB(q)))
template <int NC>
struct AdjConstsP {
    float2 hbp[4][NC];          // b_bp (feq_PA, feq_PB) in powers of phi: P = a_bp ft + hbp(phi) (Eq. 2.21)
    float2 fq[4][NC];           // (feq_PA, feq_PB)
    float2 dq[4][NC];           // (feq_PA', feq_PB') (the top coefficient is zero)
    float2 Au[2][4], Bu[2][4];  // d feq / d u_a = Au b(phi) + Bu Cint(phi) per pair (u of B = u b)
    float Au0[2], Bu0[2];       // the rest velocity's
    float bpoly[NC], cpoly[NC];
    float a_bp, b_bp, a_tp, b_tp, a_f, b_f;
    float da_bp, db_bp, da_tp, db_tp, da_f, db_f;  // d/dlambda of the weights
    float hc;
    float bcv[4];  // Dirichlet wall values W, E, S, N
};

template <int NC>
__device__ __forceinline__ F2 ap_hbp(const AdjConstsP<NC>& k, int q, F2 x) {
    F2 s{k.hbp[q][NC - 1]};
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma2(s, x, F2{k.hbp[q][m]});
    return s;
}
template <int NC>
__device__ __forceinline__ F2 ap_feq(const AdjConstsP<NC>& k, int q, F2 x) {
    F2 s{k.fq[q][NC - 1]};
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) s = fma2(s, x, F2{k.fq[q][m]});
    return s;
}
template <int NC>
__device__ __forceinline__ F2 ap_dfeq(const AdjConstsP<NC>& k, int q, F2 x) {
    F2 s{k.dq[q][NC - 2]};
#pragma unroll
    for (int m = NC - 3; m >= 0; --m) s = fma2(s, x, F2{k.dq[q][m]});
    return s;
}
__device__ __forceinline__ float hsum(F2 a) { return a.v.x + a.v.y; }
__device__ __forceinline__ float hdot(F2 a, F2 b) { return fmaf(a.v.x, b.v.x, a.v.y * b.v.y); }

// du[a] += b(phi) sum_q w_q . Au[a][q] + Cint(phi) sum_q w_q . Bu[a][q] over the pairs in
// qmask (bit q), plus the rest velocity weighted by wz (a row's sum, added in FP64 per row)
template <int NC>
__device__ __forceinline__ void ap_add_du(const AdjConstsP<NC>& k, float phi, const F2 (&w)[4], unsigned qmask,
                                          float wz, float (&du)[2]) {
    float bv = k.bpoly[NC - 1], cv = k.cpoly[NC - 1];
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) {
        bv = fmaf(bv, phi, k.bpoly[m]);
        cv = fmaf(cv, phi, k.cpoly[m]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        F2 sa = f2(0.f), sb = f2(0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (qmask & (1u << q)) {
                sa = fma2(w[q], F2{k.Au[a][q]}, sa);
                sb = fma2(w[q], F2{k.Bu[a][q]}, sb);
            }
        const float ta = fmaf(wz, k.Au0[a], hsum(sa)), tb = fmaf(wz, k.Bu0[a], hsum(sb));
        du[a] += fmaf(bv, ta, cv * tb);
    }
}

// Mirrored NEE ghost beyond a Dirichlet wall with value bv: P_g = feq(phi_g) + P_c - feq(phi_c),
// phi_g = 2 bv - phi_c, of the interior cell c it mirrors (ftilde ft).  P (in) is P_c; returns
// the ghost's zeroth moment phi_g.
template <int NC>
__device__ __forceinline__ float ap_ghost(const AdjConstsP<NC>& k, const float phc, const float bv, V9& P) {
    const float phg = 2.f * bv - phc;
    const F2 xc = f2(phc), xg = f2(phg);
    F2 s = f2(0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const F2 d = ap_feq(k, q, xg) - ap_feq(k, q, xc);
        P.p[q] = P.p[q] + d;
        s = s + d;
    }
    P.z += (phg - phc) - hsum(s);  // rest velocity: zeroth moment
    return phg;
}

// The adjoint B of such a ghost folded back into its interior cell (ftilde ft): v = the
// addition to lam of the cell (transposes of Eq. 2.21 and of phi = sum f through both
// equilibria); its dJ/dlambda and dJ/du terms are added to rl, ru.
template <int NC, bool WU>
__device__ __forceinline__ void ap_ghost_fold(const AdjConstsP<NC>& k, const V9& B, const V9& ft, const float bv,
                                              V9& v, float& rl, float (&ru)[2]) {
    const float phc = vsum(ft), phg = 2.f * bv - phc;
    const F2 xc = f2(phc), xg = f2(phg);
    const F2 c1 = f2(k.b_bp - 1.f);
    F2 pb = f2(0.f), dcs = f2(0.f), dgs = f2(0.f), fcs = f2(0.f), sp = f2(0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const F2 dc = ap_dfeq(k, q, xc), dg = ap_dfeq(k, q, xg), fc = ap_feq(k, q, xc);
        pb = fma2(B.p[q], fma2(c1, dc, f2(-1.f) * dg), pb);
        dcs = dcs + dc;
        dgs = dgs + dg;
        fcs = fcs + fc;
        sp = fma2(B.p[q], fma2(f2(k.da_bp), ft.p[q], f2(k.db_bp) * fc), sp);
    }
    // the rest velocity's derivatives and equilibrium follow the zeroth moment
    const float dc0 = 1.f - hsum(dcs), dg0 = 1.f - hsum(dgs), fc0 = phc - hsum(fcs);
    const float phibar = fmaf(B.z, fmaf(k.b_bp - 1.f, dc0, -dg0), hsum(pb));
    const F2 ph2 = f2(phibar);
#pragma unroll
    for (int q = 0; q < 4; ++q) v.p[q] = fma2(f2(k.a_bp), B.p[q], ph2);
    v.z = fmaf(k.a_bp, B.z, phibar);
    rl += hsum(sp) + B.z * fmaf(k.da_bp, ft.z, k.db_bp * fc0);
    if (WU) {  // (b_bp - 1) feq(phi_c) and feq(phi_g) in P_g
        F2 w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = c1 * B.p[q];
        ap_add_du(k, phc, w, 0xFu, (k.b_bp - 1.f) * B.z, ru);
        F2 wg[4] = {B.p[0], B.p[1], B.p[2], B.p[3]};
        ap_add_du(k, phg, wg, 0xFu, B.z, ru);
    }
}

// S: ring stages (a power of two keeps the stage index a mask); WU: also form the u-derivative;
// WALL: the grid has a Dirichlet wall on some axis (mirrored NEE ghosts, their adjoints folded
// back into the cells they mirror; else both axes are periodic)
template <int NC, int S, bool WU, bool WALL>
__global__ void __launch_bounds__(32, WALL ? DUGKS_ADJ_ROWS_WALL_MIN_WARPS : DUGKS_ADJ_ROWS_MIN_WARPS)
    adj_rows_kernel(const __grid_constant__ CUtensorMap tf, const __grid_constant__ CUtensorMap tmu,
                    const StepArgs<float, NC> a, const AdjConstsP<NC> k, const AdjArgs<float> g,
                    const int seg_rows) {
    static_assert(S >= 3 && (S & (S - 1)) == 0, "the ring holds rows n - 2 .. n; a power of two");
    using L = AdjRowLayout;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* stages = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(stages + size_t(S) * L::STAGE_BYTES);
    const int lane = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int xw = blockIdx.x * L::WI;
    const int y0 = blockIdx.y * seg_rows;
    if (y0 >= ny || xw >= nx) return;
    const int y1 = min(y0 + seg_rows, ny);
    const long long cplane = (long long)nx * ny;
    const int j = xw - 2 + lane;                // this lane's column (periodic image when outside)
    const int jw = ((j % nx) + nx) % nx;
    const int xs = (xw - 2) & ~3;               // 16-byte aligned x of the box
    const bool XW = WALL && !a.xper, YW = WALL && !a.yper;  // Dirichlet walls in x, in y
    // with x-walls every lane reads the box: a ghost column (j = -1, nx) the ftilde of the cell it
    // mirrors, a column beyond the ghosts the nearest cell's (zero weights only), and mu at its own
    // column, which the TMA zero fill makes 0 outside the domain
    const bool from_smem = XW || (j >= 0 && j < nx);  // else read the periodic image from global memory
    const bool gcol = XW && (j == -1 || j == nx);
    const int jf = XW ? min(max(j, 0), nx - 1) : j;   // column of this lane's ftilde
    const bool owner = lane >= 2 && lane <= 29 && j < nx;
    const bool xedge = XW && (xw - 2 <= -1 || xw + 29 >= nx);  // the strip holds a ghost column
    const int R = y1 - y0 + 4;                  // rows y0-2 .. y1+1
    auto wrow = [&](int r) { return r < 0 ? r + ny : (r >= ny ? r - ny : r); };  // r in [-3, ny + 1], ny >= 4
    // rows: ftilde (a ghost row the row it mirrors), mu (outside the domain: the TMA zero fill) and
    // the cell-metric row (ghost rows carry zero metrics)
    auto frow = [&](int r) { return YW ? min(max(r, 0), ny - 1) : wrow(r); };
    auto mrow = [&](int r) { return YW ? r : wrow(r); };
    auto crow = [&](int r) { return YW ? min(max(r, -1), ny) : wrow(r); };

    // this lane's cell: its east face (it is the left cell) and its west face (the right cell)
    const int jm = XW ? min(max(j, -1), nx) : jw;
    const FaceM<float> fE = a.fx[jm + 2], fW = a.fx[jm + 1];
    const CellM<float> cxj = a.cx[jm + 1];
    const float hx_e = k.hc * fE.tl, hx_w = k.hc * fW.tr;  // weights of this cell's y-slope at the two faces
    const float mhig = -k.hc * cxj.ig;                     // x-slope factor of this cell at its y-faces

    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](int t) {  // row y0 - 2 + t into stage t % S
        const int st = t & (S - 1), r = y0 - 2 + t;
        mbar_arrive_expect_tx(&bars[st], uint32_t(2 * L::BOX_BYTES));
        tma_load_3d(stages + size_t(st) * L::STAGE_BYTES, &tf, &bars[st], xs, frow(r), 0);
        tma_load_3d(stages + size_t(st) * L::STAGE_BYTES + L::MU_OFF, &tmu, &bars[st], xs, mrow(r), 0);
    };
    if (lane == 0)
        for (int t = 0; t < min(S, R); ++t) issue(t);
    // row r's ftilde (which = 0) or mu (1) as pairs: stage of row r, or the periodic image in global memory
    auto row_v9 = [&](int r, int which, V9& v) {
        const int t = r - (y0 - 2);
        if (from_smem) {
            const float* st = reinterpret_cast<const float*>(stages + size_t(t & (S - 1)) * L::STAGE_BYTES +
                                                             (which ? L::MU_OFF : 0)) + ((which ? j : jf) - xs);
            v.z = st[0];
#pragma unroll
            for (int q = 0; q < 4; ++q) v.p[q] = f2(st[PA(q) * L::BOXW], st[PB(q) * L::BOXW]);
        } else if (which && YW && (r < 0 || r >= ny)) {  // mu outside the domain
            v.z = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) v.p[q] = f2(0.f);
        } else {
            const float* src = (which ? g.mu : g.f) + (long long)(which ? wrow(r) : frow(r)) * nx + jw;
            v.z = src[0];
#pragma unroll
            for (int q = 0; q < 4; ++q) v.p[q] = f2(src[PA(q) * cplane], src[PB(q) * cplane]);
        }
    };

    V9 Pm2, Pm1, Pn;  // P = fbar^+ of rows n-2, n-1, n (this lane's column)
    V9 Ba, Bb, Bc;    // adjoint of P accumulated for rows n-2, n-1, n
#pragma unroll
    for (int q = 0; q < 4; ++q) Pm2.p[q] = Pm1.p[q] = Ba.p[q] = Bb.p[q] = Bc.p[q] = f2(0.f);
    Pm2.z = Pm1.z = Ba.z = Bb.z = Bc.z = 0.f;
    float ph1 = 0.f, mx1 = 0.f, my1 = 0.f, my2 = 0.f;  // moments: phi, Mx of row n-1; My of rows n-1, n-2
    F2 gx1[2] = {f2(0.f), f2(0.f)};                     // x-slopes of P of row n-1 (pairs 2, 3)
    float gmx1 = 0.f;                                   // x-slope of Mx of row n-1
    double djdl = 0.0, du[2] = {0.0, 0.0};
    bool failed = false;
    int t = 0;
    for (; t < R; ++t) {
        const int n = y0 - 2 + t;
        // row metrics, loaded before the wait: ig of row n - 1 (x-faces), r of rows n - 1, n and
        // the y-face below row n
        const float igq = a.cy[crow(n - 1) + 1].ig;
        const float rL = a.cy[crow(n - 1) + 1].r, rR = a.cy[crow(n) + 1].r;
        const FaceM<float> m = a.fy[min(max(n, -1), ny + 1) + 1];
        float rl = 0.f, ru[2] = {0.f, 0.f};  // this row's dJ/dlambda and dJ/du terms (FP32), added in FP64
        const bool ok = mbar_wait_bounded(&bars[t & (S - 1)], uint32_t((t / S) & 1), 2000000000ull);
        if (__any_sync(0xffffffffu, !ok)) { failed = true; break; }
        // P of the new row (Eq. 2.21; periodic, no ghosts), its moments and x-slopes
        float phn;
        {
            V9 F;
            row_v9(n, 0, F);
            phn = vsum(F);
            const F2 x2 = f2(phn);
            F2 hs = f2(0.f);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const F2 h = ap_hbp(k, q, x2);
                Pn.p[q] = fma2(f2(k.a_bp), F.p[q], h);
                hs = hs + h;
            }
            Pn.z = fmaf(k.a_bp, F.z, fmaf(k.b_bp, phn, -hsum(hs)));  // rest velocity: zeroth moment
            if constexpr (WALL) {  // mirrored ghosts (corner ghosts, never used, kept at zero)
                const bool grow = YW && (n == -1 || n == ny);
                if (gcol && grow) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) Pn.p[q] = f2(0.f);
                    Pn.z = 0.f;
                    phn = 0.f;
                } else if (gcol || grow) {
                    phn = ap_ghost(k, phn, gcol ? (j < 0 ? k.bcv[0] : k.bcv[1]) : (n < 0 ? k.bcv[2] : k.bcv[3]), Pn);
                }
            }
        }
        const float d0 = Pn.p[0].v.x - Pn.p[0].v.y, d1 = Pn.p[1].v.x - Pn.p[1].v.y;
        const float d2 = Pn.p[2].v.x - Pn.p[2].v.y, d3 = Pn.p[3].v.x - Pn.p[3].v.y;
        const float mxn = (d0 + d2) - d3, myn = (d1 + d2) + d3;  // e_x, e_y of the pairs' first velocities
        const F2 igx2 = f2(cxj.ig);
        const F2 gxn[2] = {(shfl_dn2(Pn.p[2]) - shfl_up2(Pn.p[2])) * igx2,
                           (shfl_dn2(Pn.p[3]) - shfl_up2(Pn.p[3])) * igx2};
        const float gmxn = (__shfl_down_sync(0xffffffffu, mxn, 1) - __shfl_up_sync(0xffffffffu, mxn, 1)) * cxj.ig;

        V9 mq;  // mu of row n - 1
        if (n >= y0) {
            // x-faces of row n - 1 (rows y0-1 .. y1); crossing pairs 0, 2, 3 in slots 0, 1, 2
            row_v9(n - 1, 1, mq);
            F2 fb[3];
            float phib;
            {
                // this lane's half of its east face (left cell) and of its west face (right cell)
                F2 hl[3], hr[3];
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    const int q = s == 0 ? 0 : s + 1;
                    hl[s] = sgn2(1.f - fE.w, fE.hcd, QX(q)) * Pm1.p[q];
                    hr[s] = sgn2(fW.w, -fW.hcd, QX(q)) * Pm1.p[q];
                    if (q != 0) {  // e_y = (+1, -1): the tangential term -e_y hc t G
                        const F2 gy = (Pn.p[q] - Pm2.p[q]) * f2(igq);
                        hl[s] = fma2(f2(-hx_e, hx_e), gy, hl[s]);
                        hr[s] = fma2(f2(-hx_w, hx_w), gy, hr[s]);
                    }
                }
                const float gmy = (myn - my2) * igq;  // y-slope of My
                const float pl = fmaf(1.f - fE.w, ph1, fmaf(fE.hcd, mx1, -hx_e * gmy));
                const float pr = fmaf(fW.w, ph1, -fmaf(fW.hcd, mx1, hx_w * gmy));
#pragma unroll
                for (int s = 0; s < 3; ++s) fb[s] = hl[s] + shfl_dn2(hr[s]);
                phib = pl + __shfl_down_sync(0xffffffffu, pr, 1);
            }
            // adjoint of the face's f (Eq. 2.12 flux): e_x (r_R mu_R - r_L mu_L)
            F2 gv[3];
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const int q = s == 0 ? 0 : s + 1;
                const F2 rm = mq.p[q] * f2(float(QX(q)) * cxj.r, -float(QX(q)) * cxj.r);
                gv[s] = shfl_dn2(rm) - rm;
            }
            // Eq. 2.22 transposed: A = a_f gv + b_f sum_m gv_m feq_m'(phi_b)
            const F2 pb2 = f2(phib);
            F2 sgp = f2(0.f), sdp = f2(0.f);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const int q = s == 0 ? 0 : s + 1;
                const F2 fe = ap_feq(k, q, pb2);
                sgp = fma2(gv[s], ap_dfeq(k, q, pb2), sgp);
                sdp = fma2(gv[s], fma2(f2(k.da_f), fb[s], f2(k.db_f) * fe), sdp);
            }
            const float sg = hsum(sgp), bsg = k.b_f * sg;
            // (with an x-wall the ghost lane j = -1 counts the wall face west of column 0)
            if ((owner || (XW && j == -1)) && n - 1 >= y0 && n - 1 < y1) {
                rl += hsum(sdp);
                if (WU) {  // Eq. 2.22: b_f feq(phi_b) of the crossing velocities
                    F2 w[4];
                    w[1] = f2(0.f);
#pragma unroll
                    for (int s = 0; s < 3; ++s) w[s == 0 ? 0 : s + 1] = f2(k.b_f) * gv[s];
                    ap_add_du(k, phib, w, 0xDu, 0.f, ru);
                }
            }
            // the face's A at its right cell (the lane to the east)
            const float bsgW = k.b_f * __shfl_up_sync(0xffffffffu, sg, 1);
            F2 A[3], AW[3];
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                A[s] = fma2(f2(k.a_f), gv[s], f2(bsg));
                AW[s] = fma2(f2(k.a_f), shfl_up2(gv[s]), f2(bsgW));
            }
            // normal weights into row n - 1; pair 1 and the rest velocity do not cross (A = b_f sg)
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const int q = s == 0 ? 0 : s + 1;
                Bb.p[q] = fma2(sgn2(1.f - fE.w, fE.hcd, QX(q)), A[s], Bb.p[q]);
                Bb.p[q] = fma2(sgn2(fW.w, -fW.hcd, QX(q)), AW[s], Bb.p[q]);
            }
            const float nz = fmaf(1.f - fE.w, bsg, fW.w * bsgW);
            Bb.p[1] = Bb.p[1] + f2(nz);
            Bb.z += nz;
            // this cell's y-slope (rows n and n - 2) at both faces: pairs 1, 2, 3 (e_y = +1, -1)
            const float mig = -igq;
            {
                const float tt = mig * fmaf(hx_e, bsg, hx_w * bsgW);
                const F2 t1 = f2(tt, -tt);
                Bc.p[1] = Bc.p[1] + t1;
                Ba.p[1] = Ba.p[1] - t1;
            }
#pragma unroll
            for (int s = 1; s < 3; ++s) {
                const F2 T = fma2(f2(hx_e), A[s], f2(hx_w) * AW[s]) * f2(mig, -mig);
                Bc.p[s + 1] = Bc.p[s + 1] + T;
                Ba.p[s + 1] = Ba.p[s + 1] - T;
            }
        }
        if (n >= y0 && n <= y1) {
            // y-face between rows n - 1 and n of this lane's column (faces y0 .. y1); crossing
            // pairs 1, 2, 3 (e_y = +1 for the first velocity) in slots 0, 1, 2
            V9 mn;
            row_v9(n, 1, mn);
            F2 fb[3], gv[3];
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const int q = s + 1;
                F2 v = fma2(sgn2(1.f - m.w, m.hcd, 1), Pm1.p[q], sgn2(m.w, -m.hcd, 1) * Pn.p[q]);
                if (q >= 2) {  // e_x = QX(q) of the first velocity: the tangential term -e_x hc (tl G_L + tr G_R)
                    const F2 gt = fma2(f2(m.tl), gx1[q - 2], f2(m.tr) * gxn[q - 2]);
                    v = fma2(f2(-float(QX(q)) * k.hc, float(QX(q)) * k.hc), gt, v);
                }
                fb[s] = v;
                gv[s] = fma2(mn.p[q], f2(rR, -rR), mq.p[q] * f2(-rL, rL));  // e_y (r_R mu_R - r_L mu_L)
            }
            const float phib = fmaf(1.f - m.w, ph1,
                                    fmaf(m.w, phn, fmaf(m.hcd, my1 - myn, -k.hc * fmaf(m.tl, gmx1, m.tr * gmxn))));
            const F2 pb2 = f2(phib);
            F2 sgp = f2(0.f), sdp = f2(0.f);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const F2 fe = ap_feq(k, s + 1, pb2);
                sgp = fma2(gv[s], ap_dfeq(k, s + 1, pb2), sgp);
                sdp = fma2(gv[s], fma2(f2(k.da_f), fb[s], f2(k.db_f) * fe), sdp);
            }
            const float bsg = k.b_f * hsum(sgp);
            F2 A[3];
#pragma unroll
            for (int s = 0; s < 3; ++s) A[s] = fma2(f2(k.a_f), gv[s], f2(bsg));
            if (owner && (n < y1 || (YW && n == ny))) {  // (a y-wall's top face is its own face)
                rl += hsum(sdp);
                if (WU) {
                    F2 w[4];
                    w[0] = f2(0.f);
#pragma unroll
                    for (int s = 0; s < 3; ++s) w[s + 1] = f2(k.b_f) * gv[s];
                    ap_add_du(k, phib, w, 0xEu, 0.f, ru);
                }
            }
            // normal weights into rows n - 1 (below) and n (above); pair 0 and the rest velocity
            // do not cross (A = b_f sg)
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                Bb.p[s + 1] = fma2(sgn2(1.f - m.w, m.hcd, 1), A[s], Bb.p[s + 1]);
                Bc.p[s + 1] = fma2(sgn2(m.w, -m.hcd, 1), A[s], Bc.p[s + 1]);
            }
            const float nb = (1.f - m.w) * bsg, nc = m.w * bsg;
            Bb.p[0] = Bb.p[0] + f2(nb);
            Bb.z += nb;
            Bc.p[0] = Bc.p[0] + f2(nc);
            Bc.z += nc;
            // the x-slopes of both cells (this lane's weights Z = -hc ig e_x A, transposed central
            // difference across lanes), times tl for row n - 1 and tr for row n: pairs 0, 2, 3
            {
                const float z0 = mhig * bsg;  // pair 0: e_x = (+1, -1), A = b_f sg
                const float dz = __shfl_up_sync(0xffffffffu, z0, 1) - __shfl_down_sync(0xffffffffu, z0, 1);
                const F2 d = f2(dz, -dz);
                Bb.p[0] = fma2(f2(m.tl), d, Bb.p[0]);
                Bc.p[0] = fma2(f2(m.tr), d, Bc.p[0]);
            }
#pragma unroll
            for (int s = 1; s < 3; ++s) {
                const int q = s + 1;
                const F2 Z = A[s] * f2(float(QX(q)) * mhig, -float(QX(q)) * mhig);
                const F2 d = shfl_up2(Z) - shfl_dn2(Z);
                Bb.p[q] = fma2(f2(m.tl), d, Bb.p[q]);
                Bc.p[q] = fma2(f2(m.tr), d, Bc.p[q]);
            }
        }
        if constexpr (WALL) {
            // the south ghost row -1 is complete (in Ba) one pass before row 0 is: its fold waits
            // in row 0 of lam, which this lane writes when row 0 is finished
            if (YW && y0 == 0 && n == 1 && owner) {
                V9 ft0, vs;
                row_v9(0, 0, ft0);
                ap_ghost_fold<NC, WU>(k, Ba, ft0, k.bcv[2], vs, rl, ru);
                float* out = g.lam + j;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    out[PA(q) * cplane] = vs.p[q].v.x;
                    out[PB(q) * cplane] = vs.p[q].v.y;
                }
                out[0] = vs.z;
            }
        }
        if (n >= y0 + 2) {
            // row n - 2 has every contribution: transpose Eqs. 2.21 and 2.13 and phi = sum f
            const int r = n - 2;
            V9 ft, mu;
            row_v9(r, 0, ft);
            row_v9(r, 1, mu);
            const float phi = vsum(ft);
            const F2 x2 = f2(phi);
            F2 w[4];
            F2 pb = f2(0.f), dsum = f2(0.f), fsum = f2(0.f), sp = f2(0.f);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const F2 de = ap_dfeq(k, q, x2), fe = ap_feq(k, q, x2);
                w[q] = fma2(f2(k.b_bp), Ba.p[q], f2(k.b_tp) * mu.p[q]);
                pb = fma2(w[q], de, pb);
                dsum = dsum + de;
                fsum = fsum + fe;
                sp = fma2(Ba.p[q], fma2(f2(k.da_bp), ft.p[q], f2(k.db_bp) * fe), sp);
                sp = fma2(mu.p[q], fma2(f2(k.da_tp), ft.p[q], f2(k.db_tp) * fe), sp);
            }
            const float de0 = 1.f - hsum(dsum), fe0 = phi - hsum(fsum);  // rest velocity: zeroth moment
            const float wz = fmaf(k.b_bp, Ba.z, k.b_tp * mu.z);
            const float phibar = fmaf(wz, de0, hsum(pb));
            V9 addv;  // folds of the mirrored ghosts of this cell (walls)
#pragma unroll
            for (int q = 0; q < 4; ++q) addv.p[q] = f2(0.f);
            addv.z = 0.f;
            float addl = 0.f, addu[2] = {0.f, 0.f};
            float* out = g.lam + (long long)r * nx + j;
            if constexpr (WALL) {
                if (xedge) {
                    // a ghost column's adjoint, folded by its lane, goes to the lane of the cell it
                    // mirrors: column 0 takes it from lane - 1 (j = -1), column nx - 1 from lane + 1
                    V9 vg;
#pragma unroll
                    for (int q = 0; q < 4; ++q) vg.p[q] = f2(0.f);
                    vg.z = 0.f;
                    float gl = 0.f, gu[2] = {0.f, 0.f};
                    if (gcol) ap_ghost_fold<NC, WU>(k, Ba, ft, j < 0 ? k.bcv[0] : k.bcv[1], vg, gl, gu);
                    const float fw = j == 0 ? 1.f : 0.f, fe = j == nx - 1 ? 1.f : 0.f;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        addv.p[q] = fma2(f2(fw), shfl_up2(vg.p[q]), f2(fe) * shfl_dn2(vg.p[q]));
                    addv.z = fmaf(fw, __shfl_up_sync(0xffffffffu, vg.z, 1), fe * __shfl_down_sync(0xffffffffu, vg.z, 1));
                    addl = fmaf(fw, __shfl_up_sync(0xffffffffu, gl, 1), fe * __shfl_down_sync(0xffffffffu, gl, 1));
                    if (WU)
#pragma unroll
                        for (int a2 = 0; a2 < 2; ++a2)
                            addu[a2] = fmaf(fw, __shfl_up_sync(0xffffffffu, gu[a2], 1),
                                            fe * __shfl_down_sync(0xffffffffu, gu[a2], 1));
                }
                if (YW && y1 == ny && r == ny - 1) {  // the north ghost row ny, complete in Bb
                    V9 vt;
                    ap_ghost_fold<NC, WU>(k, Bb, ft, k.bcv[3], vt, addl, addu);
#pragma unroll
                    for (int q = 0; q < 4; ++q) addv.p[q] = addv.p[q] + vt.p[q];
                    addv.z += vt.z;
                }
                if (YW && y0 == 0 && r == 0 && owner) {  // the south ghost row's fold, held in lam
#pragma unroll
                    for (int q = 0; q < 4; ++q) addv.p[q] = addv.p[q] + f2(out[PA(q) * cplane], out[PB(q) * cplane]);
                    addv.z += out[0];
                }
            }
            if (owner) {
                rl += hsum(sp) + fmaf(Ba.z, fmaf(k.da_bp, ft.z, k.db_bp * fe0), mu.z * fmaf(k.da_tp, ft.z, k.db_tp * fe0));
                if (WU) ap_add_du(k, phi, w, 0xFu, wz, ru);  // b_bp feq(phi) in P, b_tp feq(phi) in ftilde^+
                if constexpr (WALL) {
                    rl += addl;
                    if (WU) {
                        ru[0] += addu[0];
                        ru[1] += addu[1];
                    }
                }
                const F2 ph2 = f2(phibar);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const F2 l = fma2(f2(k.a_bp), Ba.p[q], fma2(f2(k.a_tp), mu.p[q], ph2)) + addv.p[q];
                    out[PA(q) * cplane] = l.v.x;
                    out[PB(q) * cplane] = l.v.y;
                }
                out[0] = fmaf(k.a_bp, Ba.z, fmaf(k.a_tp, mu.z, phibar)) + addv.z;
            }
        }
        djdl += double(rl);
        if (WU) {
            du[0] += double(ru[0]);
            du[1] += double(ru[1]);
        }
        // the stage of row n - 2 is no longer read: refill it
        __syncwarp();
        if (n >= y0 && lane == 0 && t - 2 + S < R) {
            fence_proxy_async_smem();
            issue(t - 2 + S);
        }
        Pm2 = Pm1;
        Pm1 = Pn;
        Ba = Bb;
        Bb = Bc;
#pragma unroll
        for (int q = 0; q < 4; ++q) Bc.p[q] = f2(0.f);
        Bc.z = 0.f;
        my2 = my1;
        my1 = myn;
        ph1 = phn;
        mx1 = mxn;
        gmx1 = gmxn;
        gx1[0] = gxn[0];
        gx1[1] = gxn[1];
    }
    if (failed && lane == 0) {
        atomicOr(a.err, 1);
        // let the copies still in flight land before the warp exits: rows t .. issued - 1
        const int released = max(0, t - 2);
        const int issued = min(R, released + S);
        for (int u = t; u < issued; ++u) mbar_wait_bounded(&bars[u & (S - 1)], uint32_t((u / S) & 1), 100000000ull);
    }
    __syncwarp();
    const double v[3] = {djdl, du[0], du[1]};
    block_partial3(v, g.partial + blockIdx.y * gridDim.x + blockIdx.x, g.pstride, g.accumulate);
}

}  // namespace dugks
